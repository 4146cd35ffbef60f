// rom.cu -- online solve of the reduced model (Sec. workflow:MOR, Eq.
// ap4:fully_reduced) for a batch of parameter instances.
//
// The reduced residual of an instance at coefficients a is
//   Ms (a - a_old)/dt + Alin a + mu bbnd + Pbv f_bv(a) + P1c f_1c(a),
// where f_bv, f_1c are the interface and migration terms of the full-order
// residual at the empirical-interpolation points, evaluated on the
// reconstruction u_loc = U_loc a over the stencil closure of the points (the
// voxels and faces those rows depend on).  Each point is described on the
// host by a short "term program": the faces that feed its row (interface
// faces with their row weights for the Butler-Volmer / counter-electrode and
// the plating current, electrolyte faces for the migration term) with the
// closure slots of their unknowns.  Per Newton iteration and instance:
//   gather u_loc = U_loc a; evaluate f and its sparse derivative rows G;
//   GU = G U_loc; J = Ms/dt + Alin + P GU; r as above; solve J delta = -r by
//   LU with partial pivoting after row/column equilibration; step length
//   min(1, 0.25 / |U_loc delta|_s), converged at lam |U_loc delta|_s <= 1e-12
//   (or at a full step below 1e-10 that did not halve the previous one: the
//   rounding floor of the reconstruction),
//   |.|_s the max-norm with voxel slots in their scales and plated
//   inventories relative to max(n_c, |n|).
// Plating gates: the full-order rule on the reconstruction, with the
// active-set passes of the full-order step.
// Precision: the state a, the interpolated terms f and the residual are
// FP64 and the reconstruction float-float, so the converged solution is the
// FP64 one up to ~2^-44 of the reconstruction; the
// Newton matrix (GU, the contraction P GU as one GEMM over all instances on
// the tensor cores with FP32 accuracy, its LU) and the step-length norm are
// FP32 (an inexact Newton iteration: GB300's FP64 rate is a small fraction of
// its FP32 rate).  An instance escalates for the rest of its time step when
// its iteration stagnates (a full step whose norm fell by less than 10 %,
// from the third iteration of a pass) or has not converged after
// ROM_HP_AFTER iterations: an FP32 matrix cannot converge when the
// equilibrated reduced Jacobian's condition number approaches 1/eps_32 (POD
// modes kept down to tiny singular values).  Escalated: FP64 derivatives and
// G U_loc, then the Newton step by GMRES on FP64 products preconditioned by
// the instance's FP32 LU kept from its last FP32-matrix iteration (ir, the
// default), or by an FP64 Newton matrix and LU.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mb_internal.h"

namespace mb {

constexpr int TMAX = 6;          // face terms per interpolation point
constexpr int GMAX = 32;         // closure slots one point depends on
constexpr int ROM_NR_MAX = 512;  // largest reduced dimension
constexpr int ROM_MAXIT = 30;
constexpr int ROM_PASSES = 3;
constexpr double ROM_DELTA_MAX = 0.25;
constexpr double ROM_TOL = 1e-12;
constexpr double ROM_TOL_FLOOR = 1e-10;   // the full-order production tolerance (rounding-floor stop)
constexpr int RP = 4;            // per-instance parameters: I_app, s_i0, k_pl, 1/dt
constexpr int ROM_HP_AFTER = 8;  // FP32-matrix iterations of a pass before an instance switches to FP64

enum RomTerm : int8_t { T_NONE = 0, T_GE = 1, T_KE = 2, T_LE = 3, T_EE = 4 };

struct RomDev {
    int Nr = 0, Mbv = 0, M1c = 0, M = 0, nloc = 0, ngate = 0;
    int tc = 1;                // Newton-matrix GEMM on the tensor cores (3xTF32), else FP32 FMA
    int graph = 1;             // a time step as one CUDA graph (else driven from the host)
    int ir = 1;                // escalated instances: GMRES on FP64 products preconditioned by the kept FP32 LU
    double* UlocR = nullptr;   // nloc x Nr
    double* us = nullptr;      // nloc unknown scales
    int8_t* ttype = nullptr;   // M x TMAX
    int32_t* tidx = nullptr;   // M x TMAX x 5 closure slots (c_s, phi_s, c_e, phi_e, n), -1 unused
    double* twbv = nullptr;    // M x TMAX row weight of the BV / CE current (or of the migration flux)
    double* twpl = nullptr;    // M x TMAX row weight of the plating current
    int32_t* tgate = nullptr;  // M x TMAX gate slot, -1 none
    int8_t* tgpos = nullptr;   // M x TMAX x 5 position in the point's derivative list
    int32_t* gidx = nullptr;   // M x GMAX closure slots of the derivative list, -1 unused
    int32_t* gface = nullptr;  // ngate x 3 closure slots (phi_g, phi_e, n) of the gated faces
    double* P = nullptr;       // Nr x M (Pbv | P1c)
    float2* Pdf = nullptr;     // float-float copies of P, Ms, Alin: the escalated GMRES's products
    float2* Msdf = nullptr;
    float2* Alindf = nullptr;
    double* Ms = nullptr;      // Nr x Nr
    double* Alin = nullptr;    // Nr x Nr
    float* Ptf = nullptr;      // FP32 copies for the Newton matrix: P^T (M x Nr), Ms, Alin, UlocR, UlocC, us
    float* Pbf = nullptr;      // TF32 head and tail of P, the tcgen05 GEMM's B operand, stored per K
    float* Psf = nullptr;      //   slice of 32 in its shared-memory tile layout (Mpad/32 tiles of Npad x 32)
    int Npad = 0, Mpad = 0;    // Nr rounded up to 16, M rounded up to the K slice
    float* Msf = nullptr;
    float* Alinf = nullptr;
    float* UlocRf = nullptr;
    float* UlocCf = nullptr;
    float2* UlocCdf = nullptr; // Nr x nloc float-float copy for the reconstruction
    float* usf = nullptr;
    float* uscf = nullptr;     // nloc: the scales of the step-length cap (voxel slots; -1 marks face slots,
                               //   capped relative to max(n_c, |n|) of the current reconstruction)
    float ncf = 0.f;           // n_c
    double* bbnd = nullptr;    // Nr
    double* scp = nullptr;     // Nr
    double* sac = nullptr;     // Nr
    double* a0 = nullptr;      // Nr
};

struct RomWork {
    int B = 0;
    double *a = nullptr, *a_old = nullptr, *delta = nullptr, *r = nullptr;
    float* J = nullptr;        // B x Nr x Nr, instance-major
    float* GU = nullptr;       // M x B x Nr: row p of every instance's G U_loc (the GEMM's right operand)
    double *uloc = nullptr, *uloc_old = nullptr, *f = nullptr;
    float* G = nullptr;        // B x M x GMAX derivative lists (FP32: they only feed the Newton matrix)
    float* dpart = nullptr;    // B x ceil(nloc / UN_K): partial maxima of the step-length norm
    int* hp = nullptr;         // B: instance has escalated to FP64 (for the rest of the time step)
    int* pit = nullptr;        // B: iterations in the current pass
    float* dnprev = nullptr;   // B: step norm of the previous iteration
    double* G64 = nullptr;     // B x M x GMAX   FP64 derivative lists of the hp instances
    double* GU64 = nullptr;    // B x M x Nr     their G U_loc
    double* J64 = nullptr;     // B x Nr x Nr    their Newton matrices
    int* hplist = nullptr;     // B: the instances with hp (compacted at each count; order irrelevant)
    int* lpiv = nullptr;       // B x Nr   pivot rows of the kept FP32 LU factors (in J; refinement mode)
    float* lsc = nullptr;      // B x 2 Nr their row and column scales
    int* alist = nullptr;      // B: the active instances on the FP32 matrix (compacted at each count)
    int n_alist = -1;          // host: its length at the last count (-1: not counted yet: all B)
    int hp_any = 0;            // host: number of instances with hp at the last count
    double* prm = nullptr;
    uint8_t *gate = nullptr, *gate2 = nullptr;
    int *active = nullptr, *failed = nullptr, *pass_on = nullptr, *counts = nullptr;
    long long* its = nullptr;
    long long* flips = nullptr;
    double *V = nullptr, *S = nullptr;
    // one reduced time step as a CUDA graph (conditional nodes run the passes,
    // the Newton iterations and the escalated branch on the device)
    cudaGraphExec_t gexec = nullptr;
    int* ctl = nullptr;        // device: [0] Newton iteration of the pass, [1] passes done
    int* tcerr = nullptr;      // device: a bounded wait of the tcgen05 GEMM gave up
    bool graph_failed = false; // the graph could not be built: host-driven steps
    int g_tc = -1, g_ir = -1;  // the GEMM variant and escalation mode the graph was captured with
    int g_rate = -1;           // and the Newton stopping rule (newton_rate_test)
    double* a_hold = nullptr;  // B x Nr: the state before the step (dt halving restarts from it)
    int* retry = nullptr;      // B: instances retaking the step with halved dt
    std::vector<double> hprm;  // host copy of the instance parameters (RP per instance)
    std::vector<void*> bufs;
};

}  // namespace mb

namespace mb {
// Maps of the hierarchical error estimate between this model (the reduced
// one) and a validation model (mb_rom_estimate_batch), for one validation model.
struct RomEst {
    const mb_rom* val = nullptr;
    int Nv = 0;
    double* T = nullptr;       // Nv x Nr: Uv_f^T W U_f, f the field of validation mode j (row j)
    double* G = nullptr;       // 3 x Nr x Nr: R_f^T W R_f, R_f = U_f - Uv_f T_f (U_f outside span Uv_f)
    int* fld = nullptr;        // Nv: field of validation mode j (0 c, 1 phi, 2 n; -1 none)
    int gon[3] = {0, 0, 0};    // G_f has a nonzero entry
    double* est = nullptr;     // B x 3 estimates of the current step
    double* nrm = nullptr;     // B x 3 norms of the validation model's fields
    int Bcap = 0;
    std::vector<void*> bufs;
};
}  // namespace mb

struct mb_rom {
    mb_cell* cell = nullptr;
    mb::RomDev d;
    std::vector<void*> owned;
    mb::RomWork w;
    std::vector<double> hU;    // host copy of the basis (n x Nr, row-major): the error estimate's maps
    mb::RomEst est;
    bool tc_forced = false;    // the GEMM variant was set by mb_debug_rom_tensor (no autotuning)
    float tune_ms[3] = {-1.f, -1.f, -1.f};   // the last autotuning's time per variant (-1: not timed)
};

namespace mb {

static void rom_work_free(RomWork& w) {
    if (w.gexec) cudaGraphExecDestroy(w.gexec);
    for (void* p : w.bufs) cudaFree(p);
    w = RomWork();
}

// field of unknown i: 0 concentration, 1 potential, 2 plated-Li face
static inline int est_field(int64_t i, int64_t N) { return i < N ? 0 : (i < 2 * N ? 1 : 2); }

template <class T>
static T* rom_alloc(std::vector<void*>& list, size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * (n ? n : 1)) != cudaSuccess) return nullptr;
    list.push_back(p);
    return static_cast<T*>(p);
}

// ------------------------------------------------------------------ kernels
// u_loc[b] = U_loc a[b] in float-float arithmetic (products by FMA
// TwoProduct, sums by TwoSum: ~2^-46 of the terms' magnitudes, a few times
// faster than FP64 on GB300), stored as FP64
__global__ void k_rom_gather(RomDev d, const double* __restrict__ a, double* __restrict__ uloc,
                             const int* __restrict__ active) {
    __shared__ float2 sa[ROM_NR_MAX];
    const int b = blockIdx.y;
    if (active && !active[b]) return;   // a converged instance keeps its reconstruction
    for (int j = threadIdx.x; j < d.Nr; j += blockDim.x) sa[j] = df_from_double(a[(int64_t)b * d.Nr + j]);
    __syncthreads();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.nloc) return;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = 0; j < d.Nr; ++j) {
        const float2 u = d.UlocCdf[(int64_t)j * d.nloc + k], x = sa[j];
        const float p = u.x * x.x;
        float e = fmaf(u.x, x.x, -p);
        e = fmaf(u.x, x.y, fmaf(u.y, x.x, e));
        acc = df_add(acc, make_float2(p, e));
    }
    uloc[(int64_t)b * d.nloc + k] = df_to_double(acc);
}

// gate of the gated faces: plated Li present or negative plating overpotential
__global__ void k_rom_gate(RomDev d, int B, const double* __restrict__ uloc, const double* __restrict__ uloc_old,
                           double n_thr, uint8_t* __restrict__ gate) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)d.ngate * B) return;
    const int b = (int)(i / d.ngate), g = (int)(i % d.ngate);
    const double* u = uloc + (int64_t)b * d.nloc;
    const double* uo = uloc_old + (int64_t)b * d.nloc;
    const int32_t* s = d.gface + 3 * g;
    const double etap = u[s[0]] - u[s[1]];
    gate[i] = (uo[s[2]] > n_thr || etap < 0.0) ? 1 : 0;
}

// f (FP64) and its derivative list at every point, for the instances whose
// Newton-matrix precision matches HP (FP64 derivatives to G64 when HP, FP32
// to G otherwise)
template <bool HP>
__global__ void k_rom_ei(RomDev d, DevParams P, ParT<float> Pf, int B, const double* __restrict__ uloc,
                         const uint8_t* __restrict__ gate, const double* __restrict__ prm,
                         const int* __restrict__ active, const int* __restrict__ hp,
                         const int* __restrict__ hplist, double* __restrict__ f, float* __restrict__ G,
                         double* __restrict__ G64) {
    using TG = typename std::conditional<HP, double, float>::type;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)d.M * B) return;   // HP: B = length of hplist
    int b = (int)(i / d.M);
    const int p = (int)(i % d.M);
    if (HP) {
        b = hplist[b];
        if (b < 0) return;   // past the end of the list (launched for the whole batch)
    }
    if (!active[b] || (hp[b] != 0) != HP) return;
    const double* u = uloc + (int64_t)b * d.nloc;
    const double s_i0 = prm[RP * b + 1], k_pl = prm[RP * b + 2];
    TG g[GMAX];
#pragma unroll
    for (int e = 0; e < GMAX; ++e) g[e] = TG(0);
    double fv = 0.0;
    for (int t = 0; t < TMAX; ++t) {
        const int q = p * TMAX + t;
        const int type = d.ttype[q];
        if (type == T_NONE) break;
        const int32_t* sl = d.tidx + 5 * q;
        const int8_t* gp = d.tgpos + 5 * q;
        if (type == T_EE) {
            // A j_m = -E_gm (c_w - c_v) / S, S = max(c_v, cmin) + max(c_w, cmin)
            const double cv = u[sl[0]], cw = u[sl[2]], cmin = P.cmin[PE];
            const double S = fmax(cv, cmin) + fmax(cw, cmin);
            const double dc = cw - cv, gm = P.E_gm;
            const double w = d.twbv[q];
            fv += w * (-gm * dc / S);
            g[gp[0]] += (TG)(w * (gm / S + (cv >= cmin ? gm * dc / (S * S) : 0.0)));
            g[gp[2]] += (TG)(w * (-gm / S + (cw >= cmin ? gm * dc / (S * S) : 0.0)));
        } else {
            const int ls = type == T_GE ? PG : (type == T_KE ? PK : PL);
            const double cs = sl[0] >= 0 ? u[sl[0]] : 0.0, ps = u[sl[1]];
            const double ce = sl[2] >= 0 ? u[sl[2]] : 0.0, pe = u[sl[3]];
            const double nf = sl[4] >= 0 ? u[sl[4]] : 0.0;
            const bool gt = d.tgate[q] >= 0 && gate[(int64_t)b * d.ngate + d.tgate[q]] != 0;
            double ibv, ipl;
            interface_current<double>(P, ls, cs, ps, ce, pe, nf, gt, s_i0, k_pl, ibv, ipl);
            TG i_eta, i_cs, i_ce, ip_eta, ip_ce, ip_n;
            if constexpr (HP)
                interface_partials<double>(P, ls, cs, ps, ce, pe, nf, gt, s_i0, k_pl, i_eta, i_cs, i_ce, ip_eta, ip_ce,
                                           ip_n);
            else
                interface_partials<float>(Pf, ls, (float)cs, (float)ps, (float)ce, (float)pe, (float)nf, gt,
                                          (float)s_i0, (float)k_pl, i_eta, i_cs, i_ce, ip_eta, ip_ce, ip_n);
            const double wbd = d.twbv[q], wpd = d.twpl[q];
            fv += wbd * ibv + wpd * ipl;
            const TG wb = (TG)wbd, wp = (TG)wpd;
            if (sl[0] >= 0) g[gp[0]] += wb * i_cs;
            g[gp[1]] += wb * i_eta + wp * ip_eta;
            if (sl[2] >= 0) g[gp[2]] += wb * i_ce + wp * ip_ce;
            g[gp[3]] += -(wb * i_eta + wp * ip_eta);
            if (sl[4] >= 0) g[gp[4]] += wp * ip_n;
        }
    }
    f[(int64_t)b * d.M + p] = fv;
    TG* Gp;
    if constexpr (HP)
        Gp = G64 + ((int64_t)b * d.M + p) * GMAX;
    else
        Gp = G + ((int64_t)b * d.M + p) * GMAX;
#pragma unroll
    for (int e = 0; e < GMAX; ++e) Gp[e] = g[e];
}

// GU[p][b][j] = sum_e G[b][p][e] U_loc[gidx[p][e]][j] (FP32); inactive and
// escalated instances write zeros so that the GEMM reads defined values.
// One block per (point p, chunk of GU_INST instances): the point's closure
// rows of U_loc (at most GMAX x Nr) are staged in shared memory once and
// shared by the chunk's instances (read for every instance from L2 they
// made the kernel L2-bound); warps take instances, lanes the columns j.
constexpr int GU_INST = 64;
__global__ void __launch_bounds__(256) k_rom_gu(RomDev d, int B, const float* __restrict__ G,
                                                const int* __restrict__ active, const int* __restrict__ hp,
                                                float* __restrict__ GU) {
    extern __shared__ __align__(16) float gu_s[];   // ne x Nr staged rows of U_loc
    const int p = blockIdx.x, b0 = blockIdx.y * GU_INST;
    const int Nr = d.Nr;
    const int32_t* gi = d.gidx + (int64_t)p * GMAX;
    int ne = 0;
    while (ne < GMAX && gi[ne] >= 0) ++ne;
    for (int e = threadIdx.x; e < ne * Nr; e += blockDim.x) {
        const int q = e / Nr, j = e - q * Nr;
        gu_s[e] = d.UlocRf[(int64_t)gi[q] * Nr + j];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int bi = wid; bi < GU_INST; bi += nw) {
        const int b = b0 + bi;
        if (b >= B) break;
        float* out = GU + ((int64_t)p * B + b) * Nr;
        if (!active[b] || hp[b]) {
            for (int j = lane; j < Nr; j += 32) out[j] = 0.f;
            continue;
        }
        const float* Gp = G + ((int64_t)b * d.M + p) * GMAX;
        const float gl = lane < ne ? Gp[lane] : 0.f;   // the instance's derivative list, one entry per lane
        for (int j0 = 0; j0 < Nr; j0 += 32) {   // every lane takes every shuffle
            const int j = j0 + lane;
            const bool in = j < Nr;
            float acc = 0.f;
            for (int e = 0; e < ne; ++e) {
                const float ge = __shfl_sync(0xffffffffu, gl, e);
                if (in) acc = fmaf(ge, gu_s[e * Nr + j], acc);
            }
            if (in) out[j] = acc;
        }
    }
}

// Newton matrices of the listed instances as one GEMM with FP32 accuracy,
// C = P [GU_b0 | GU_b1 | ...] (Nr x M times M x nlist Nr), plus Ms/dt_b + Alin,
// written instance-major J[b][i][j].  Tile: 64 rows (blockIdx.y) x 64 columns
// (blockIdx.x) per block of 256 threads, K in slices of 32 staged in shared
// memory (P read from its K-major copy, the next slice fetched into registers
// while the current one is multiplied).  TC: eight warps of 32 x 16 results on
// the tensor cores (three TF32 products per pair, below); else FP32 FMA with
// 4 x 4 results per thread.  Column c = l Nr + j of instance b = alist[l].
constexpr int JT_ROWS = 64, JT_COLS = 64, JT_K = 32, JT_PAD = 8;

// TF32 tensor-core pieces (mma.sync m16n8k8, FP32 accumulation).  A value
// is split as big + small, both TF32 (big rounded to nearest, small the
// rounded remainder), and a product as big*big + big*small + small*big,
// which keeps about FP32 accuracy (the dropped small*small term is ~2^-22 of
// the product).
__device__ inline uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ inline void tf32_split(float x, uint32_t& big, uint32_t& small) {
    big = to_tf32(x);
    small = to_tf32(x - __uint_as_float(big));
}
__device__ inline void mma_tf32(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
template <bool TC>
__global__ void __launch_bounds__(256)
k_rom_jac(RomDev d, int B, int nlist, const int* __restrict__ alist, const double* __restrict__ prm,
          const float* __restrict__ GU, const int* __restrict__ hp, float* __restrict__ J,
          const int* __restrict__ dit, const int* __restrict__ dnlist) {
    __shared__ float As[JT_K][JT_ROWS + JT_PAD];
    __shared__ float Bs[JT_K][JT_COLS + JT_PAD];
    const int Nr = d.Nr, M = d.M;
    // device-side choice (a launch inside a graph, grid for the whole batch):
    // the first iteration of a pass takes every instance, later ones the list
    if (dit) {
        if (*dit > 0) nlist = *dnlist;
        else alist = nullptr;
    }
    // columns c = l Nr + j of the listed instances b = alist[l] (all B in order without a list)
    const int ncol = (alist ? nlist : B) * Nr;
    const int64_t gstride = (int64_t)B * Nr;   // row stride of GU
    const int c0 = blockIdx.x * JT_COLS;
    const int i0 = blockIdx.y * JT_ROWS;
    if (c0 >= ncol) return;   // the block's columns are all past the end
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    // loader: this thread fills column lq of both tiles at K rows kq + 4 m; the row of P^T
    // and the column of GU it reads are fixed over the K loop
    constexpr int LK = JT_K / 4;
    const int lq = threadIdx.x & 63, kq = threadIdx.x >> 6;
    const bool arow = i0 + lq < Nr, bcol = c0 + lq < ncol;
    int64_t boff = 0;
    if (bcol) {
        const int l = (c0 + lq) / Nr;
        boff = (int64_t)(alist ? alist[l] : l) * Nr + (c0 + lq - l * Nr);
    }
    float ra[LK], rb[LK];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int m = 0; m < LK; ++m) {
            const int k = k0 + kq + 4 * m;
            ra[m] = (arow && k < M) ? d.Ptf[(int64_t)k * Nr + i0 + lq] : 0.f;
            rb[m] = (bcol && k < M) ? GU[(int64_t)k * gstride + boff] : 0.f;
        }
    };
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
    fetch(0);
    for (int k0 = 0; k0 < M; k0 += JT_K) {
#pragma unroll
        for (int m = 0; m < LK; ++m) {
            As[kq + 4 * m][lq] = ra[m];
            Bs[kq + 4 * m][lq] = rb[m];
        }
        __syncthreads();
        if (k0 + JT_K < M) fetch(k0 + JT_K);   // next slice in flight during this one's products
        if (TC) {
            // warp (wr, wc) owns rows wr*32 + [0,32), columns wc*16 + [0,16): 2 x 2 tiles of 16 x 8
            const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
            const int wr = wid >> 2, wc = wid & 3;
#pragma unroll
            for (int ks = 0; ks < JT_K; ks += 8) {
                uint32_t ab[2][4], as_[2][4], bb[2][2], bs_[2][2];
#pragma unroll
                for (int mi = 0; mi < 2; ++mi) {
                    const int r0 = wr * 32 + mi * 16;
                    tf32_split(As[ks + t][r0 + g], ab[mi][0], as_[mi][0]);
                    tf32_split(As[ks + t][r0 + g + 8], ab[mi][1], as_[mi][1]);
                    tf32_split(As[ks + t + 4][r0 + g], ab[mi][2], as_[mi][2]);
                    tf32_split(As[ks + t + 4][r0 + g + 8], ab[mi][3], as_[mi][3]);
                }
#pragma unroll
                for (int ni = 0; ni < 2; ++ni) {
                    const int cb = wc * 16 + ni * 8;
                    tf32_split(Bs[ks + t][cb + g], bb[ni][0], bs_[ni][0]);
                    tf32_split(Bs[ks + t + 4][cb + g], bb[ni][1], bs_[ni][1]);
                }
#pragma unroll
                for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                    for (int ni = 0; ni < 2; ++ni) {
                        float(&cc)[4] = acc[mi * 2 + ni];
                        mma_tf32(cc, as_[mi], bb[ni]);
                        mma_tf32(cc, ab[mi], bs_[ni]);
                        mma_tf32(cc, ab[mi], bb[ni]);
                    }
            }
        } else {
#pragma unroll
            for (int k = 0; k < JT_K; ++k) {
                float a[4], bq[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) a[r] = As[k][ty * 4 + r];
#pragma unroll
                for (int q = 0; q < 4; ++q) bq[q] = Bs[k][tx * 4 + q];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(a[r], bq[q], acc[r][q]);
            }
        }
        __syncthreads();
    }
    // result element (r, q) of this thread: row and column within the tile
    auto row_of = [&](int r, int q) -> int {
        if (!TC) return ty * 4 + r;
        const int wid = threadIdx.x >> 5, g = (threadIdx.x & 31) >> 2;
        return (wid >> 2) * 32 + (r >> 1) * 16 + g + ((q >> 1) ? 8 : 0);
    };
    auto col_of = [&](int r, int q) -> int {
        if (!TC) return tx * 4 + q;
        const int wid = threadIdx.x >> 5, t = threadIdx.x & 3;
        return (wid & 3) * 16 + (r & 1) * 8 + 2 * t + (q & 1);
    };
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = c0 + col_of(r, q);
            const int i = i0 + row_of(r, q);
            if (c >= ncol || i >= Nr) continue;
            const int l = c / Nr, j = c - l * Nr;
            const int b = alist ? alist[l] : l;
            if (hp[b]) continue;   // escalated: J[b] keeps the LU factors of its last FP32 iteration
            const float dt_inv = (float)prm[RP * b + 3];
            J[((int64_t)b * Nr + i) * Nr + j] =
                acc[r][q] + d.Msf[(int64_t)i * Nr + j] * dt_inv + d.Alinf[(int64_t)i * Nr + j];
        }
}


// ---- the same Newton-matrix GEMM on the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulator in tensor memory).  One CTA of 128
// threads computes C^T for 128 GEMM columns (the MMA's M = TMEM lanes) and all
// N_r rows (the MMA's N = TMEM columns, N_r padded to a multiple of 16 <= 256):
// D[m][n] = sum_k GU[k][c0 + m] P[n][k].  K in slices of T5_K staged in shared
// memory in the no-swizzle K-major layout of 8-row x 16-byte core matrices
// (row r, element k at (k/4) LBO + (r/8) 128 + (r%8) 16 + (k%4) 4 bytes, LBO =
// rows x 16), each operand as a TF32 head and tail (the 3xTF32 split of the
// mma.sync kernel: small*big + big*small + big*big per K step), the P head and
// tail precomputed once per model directly in that tile layout, one
// contiguous N_pad x 32 tile per K slice (Pbf, Psf), so that each slice's B
// tiles arrive by two bulk asynchronous copies (cp.async.bulk, completion
// counted in bytes on an mbarrier).  One thread issues the copies and the
// MMAs; the MMAs' completion is signalled on an mbarrier by tcgen05.commit.
// Every wait is bounded: on a timeout the CTA sets *err, waits (bounded) for
// its copies and MMAs in flight, frees its tensor memory and returns.
constexpr int T5_M = 128, T5_K = 32, T5_THREADS = 256, T5_NMAX = 256;
constexpr int T5_SPIN = 1 << 22;
constexpr int T5_A_BYTES = T5_M * T5_K * 4;            // one A tile (16 KB)
constexpr int T5_B_BYTES = T5_NMAX * T5_K * 4;         // one B tile (32 KB)
constexpr int T5_TILES = 2 * T5_A_BYTES + 2 * T5_B_BYTES;   // 96 KB per pipeline stage (two stages)
// the CTA's shared memory is padded well beyond the tiles, so that no
// descriptor offset of the layout above can leave the allocation
constexpr int T5_SMEM = 225 * 1024;

__device__ inline uint32_t t5_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (8-row-group) byte offsets, descriptor version 1, no swizzle
__device__ inline uint64_t t5_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t t5_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ inline void t5_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ inline void t5_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(t5_smem(bar))
                 : "memory");
}
__device__ inline void t5_mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(t5_smem(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ inline bool t5_wait(uint64_t* bar, uint32_t parity) {
    for (int i = 0; i < T5_SPIN; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(t5_smem(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ inline void t5_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// TF32 head and tail of P for the tcgen05 GEMM's B operand, from its K-major
// FP32 copy Ptf (M x Nr), zero padded to Npad x Mpad and stored tile by tile:
// element (n, k) of K slice s = k / 32 at s Npad 32 + the byte offset
// (k%32 / 4) (Npad 16) + (n/8) 128 + (n%8) 16 + (k%4) 4 of the kernel's layout
__global__ void k_rom_psplit(int Nr, int M, int Npad, int Mpad, const float* __restrict__ Ptf,
                             float* __restrict__ Pbf, float* __restrict__ Psf) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)Npad * Mpad) return;
    const int n = (int)(e / Mpad), k = (int)(e % Mpad);
    uint32_t hb = 0u, hs = 0u;
    if (n < Nr && k < M) tf32_split(Ptf[(int64_t)k * Nr + n], hb, hs);
    const int sl = k / T5_K, kk = k % T5_K;
    const int64_t o = (int64_t)sl * Npad * T5_K +
                      ((int64_t)(kk >> 2) * Npad * 16 + (n >> 3) * 128 + (n & 7) * 16 + (kk & 3) * 4) / 4;
    Pbf[o] = __uint_as_float(hb);
    Psf[o] = __uint_as_float(hs);
}

__device__ inline void t5_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(t5_smem(bar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy of `bytes` (16-byte aligned, a multiple of 16), counted on bar
__device__ inline void t5_bulk(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(t5_smem(dst)), "l"(src), "r"(bytes), "r"(t5_smem(bar))
                 : "memory");
}

__global__ void __launch_bounds__(T5_THREADS, 1)
k_rom_jac5(RomDev d, int B, int nlist, const int* __restrict__ alist, const double* __restrict__ prm,
           const float* __restrict__ GU, const int* __restrict__ hp, float* __restrict__ J,
           const int* __restrict__ dit, const int* __restrict__ dnlist, int* __restrict__ err) {
    // Two pipeline stages of (A head, A tail, B head, B tail) tiles: while the
    // tensor core runs the MMAs of slice k - 1 from one stage, the CTA fills
    // the other with slice k (B: two bulk copies of the precomputed P head and
    // tail tiles, issued first; A: the 128 column owners split their
    // prefetched GU values into TF32 head and tail), then the prefetch of
    // slice k + 1 goes out.  A stage is refilled only after the commit of the
    // MMAs that read it (slice k - 2) has arrived on its mbarrier.
    extern __shared__ __align__(1024) uint8_t t5_raw[];
    __shared__ __align__(8) uint64_t bar[2];    // MMA completion per stage
    __shared__ __align__(8) uint64_t barb[2];   // B-tile arrival per stage
    __shared__ uint32_t tmem_slot;
    __shared__ int s_ok;   // thread 0's bounded wait, broadcast (every thread leaves the loop together)
    const int Nr = d.Nr, M = d.M, NP = d.Npad;
    const uint32_t tile_b = (uint32_t)NP * T5_K * 4;   // bytes of one B tile (head or tail)
    if (dit) {
        if (*dit > 0) nlist = *dnlist;
        else alist = nullptr;
    }
    const int ncol = (alist ? nlist : B) * Nr;
    const int64_t gstride = (int64_t)B * Nr;
    const int c0 = blockIdx.x * T5_M;
    if (c0 >= ncol) return;
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool owner = tid < T5_M;   // owns GEMM column c0 + tid (its A row)
    const uint32_t lbo_a = T5_M * 16, lbo_b = (uint32_t)NP * 16;
    if (tid == 0) {
        t5_mbar_init(&bar[0]);
        t5_mbar_init(&bar[1]);
        t5_mbar_init(&barb[0]);
        t5_mbar_init(&barb[1]);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(t5_smem(&tmem_slot)),
                     "r"(T5_NMAX));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const int c = c0 + tid;
    const bool cvalid = owner && c < ncol;
    int64_t boff = 0;
    if (cvalid) {
        const int l = c / Nr;
        boff = (int64_t)(alist ? alist[l] : l) * Nr + (c - l * Nr);
    }
    const uint32_t idesc = t5_idesc(T5_M, NP);
    bool ok = true;
    int bcopy = -1;   // a slice whose B copies may still be in flight after a timeout
    const int nsl = (M + T5_K - 1) / T5_K;
    float ra[T5_K];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int kk = 0; kk < T5_K; ++kk) {
            const int k = k0 + kk;
            ra[kk] = (cvalid && k < M) ? GU[(int64_t)k * gstride + boff] : 0.f;
        }
    };
    if (owner) fetch(0);
    int k = 0;
    for (; k < nsl; ++k) {
        const int st = k & 1;
        uint8_t* const Ab = t5_raw + st * T5_TILES;
        uint8_t* const As = Ab + T5_A_BYTES;
        uint8_t* const Bb = Ab + 2 * T5_A_BYTES;
        uint8_t* const Bs = Bb + T5_B_BYTES;
        // the MMAs of slice k - 2 have read this stage (thread 0 waits, bounded)
        if (k >= 2) {
            if (tid == 0) s_ok = t5_wait(&bar[st], (uint32_t)((k - 2) >> 1) & 1u) ? 1 : 0;
            __syncthreads();
            if (!s_ok) { ok = false; break; }
        }
        if (tid == 0) {   // B tiles of slice k: bulk copies counted on barb[st]
            t5_expect_tx(&barb[st], 2u * tile_b);
            t5_bulk(Bb, d.Pbf + (int64_t)k * NP * T5_K, tile_b, &barb[st]);
            t5_bulk(Bs, d.Psf + (int64_t)k * NP * T5_K, tile_b, &barb[st]);
        }
        if (owner) {
#pragma unroll
            for (int q = 0; q < T5_K / 4; ++q) {
                uint32_t hb[4], hs[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) tf32_split(ra[4 * q + e], hb[e], hs[e]);
                const uint32_t off = (uint32_t)q * lbo_a + (uint32_t)(tid >> 3) * 128u + (uint32_t)(tid & 7) * 16u;
                *reinterpret_cast<uint4*>(Ab + off) = make_uint4(hb[0], hb[1], hb[2], hb[3]);
                *reinterpret_cast<uint4*>(As + off) = make_uint4(hs[0], hs[1], hs[2], hs[3]);
            }
        }
        if (tid == 0) s_ok = t5_wait(&barb[st], (uint32_t)(k >> 1) & 1u) ? 1 : 0;   // the B tiles have landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (!s_ok) {
            ok = false;
            bcopy = k;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int s = 0; s < T5_K / 8; ++s) {
                const uint32_t ka = (uint32_t)(2 * s) * lbo_a, kb = (uint32_t)(2 * s) * lbo_b;
                const uint64_t dab = t5_desc(t5_smem(Ab) + ka, lbo_a, 128), das = t5_desc(t5_smem(As) + ka, lbo_a, 128);
                const uint64_t dbb = t5_desc(t5_smem(Bb) + kb, lbo_b, 128), dbs = t5_desc(t5_smem(Bs) + kb, lbo_b, 128);
                t5_mma(tmem, das, dbb, idesc, (k > 0 || s > 0) ? 1u : 0u);
                t5_mma(tmem, dab, dbs, idesc, 1u);
                t5_mma(tmem, dab, dbb, idesc, 1u);
            }
            t5_commit(&bar[st]);
        }
        if (owner && k + 1 < nsl) fetch((k + 1) * T5_K);   // the next slice in flight during the MMAs
    }
    // every MMA has completed once the last slice's commit has arrived (a commit
    // tracks all earlier tcgen05 operations of the issuing thread)
    const int last = ok ? nsl - 1 : k - 1;
    if (ok && nsl > 0) {
        if (tid == 0) s_ok = t5_wait(&bar[last & 1], (uint32_t)(last >> 1) & 1u) ? 1 : 0;
        __syncthreads();
        ok = s_ok != 0;
    }
    if (!ok) {
        if (tid == 0) {
            atomicOr(err, 1);
            if (last >= 0) t5_wait(&bar[last & 1], (uint32_t)(last >> 1) & 1u);   // bounded: the MMAs in flight
            if (bcopy >= 0) t5_wait(&barb[bcopy & 1], (uint32_t)(bcopy >> 1) & 1u);   // bounded: the copies
        }
    } else if (warp < 4) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: warp w reads TMEM lanes 32w.. (its 32 columns), 16 rows per load
        const int l = cvalid ? c / Nr : 0, j = c - l * Nr;
        const int b = cvalid ? (alist ? alist[l] : l) : 0;
        const bool wr = cvalid && !hp[b];   // escalated: J[b] keeps the LU factors of its last FP32 iteration
        const float dt_inv = wr ? (float)prm[RP * b + 3] : 0.f;
        for (int n0 = 0; n0 < NP; n0 += 16) {
            float v[16];
            t5_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0, v);
            if (wr) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int i = n0 + q;
                    if (i < Nr)
                        J[((int64_t)b * Nr + i) * Nr + j] =
                            v[q] + d.Msf[(int64_t)i * Nr + j] * dt_inv + d.Alinf[(int64_t)i * Nr + j];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T5_NMAX));
}

// host: prepare the tcgen05 GEMM's P operand and its shared memory (false:
// this model cannot use it, N_r > 256)
static bool t5_prepare(RomDev& d, std::vector<void*>& owned) {
    if (d.Nr > T5_NMAX || d.M < 1) return false;
    d.Npad = (d.Nr + 15) / 16 * 16;
    d.Mpad = (d.M + T5_K - 1) / T5_K * T5_K;
    const size_t n = (size_t)d.Npad * d.Mpad;
    d.Pbf = rom_alloc<float>(owned, n);
    d.Psf = rom_alloc<float>(owned, n);
    if (!d.Pbf || !d.Psf) return false;
    if (cudaFuncSetAttribute(k_rom_jac5, cudaFuncAttributeMaxDynamicSharedMemorySize, T5_SMEM) != cudaSuccess)
        return false;
    k_rom_psplit<<<(unsigned)((n + 255) / 256), 256>>>(d.Nr, d.M, d.Npad, d.Mpad, d.Ptf, d.Pbf, d.Psf);
    return cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
}

// FP64 Newton matrix of the instances with hp[b]: GU64[b][p][:] = G64[b][p] U_loc
// (one block per point and instance), then J64[b] = Ms/dt + Alin + P GU64[b]
// (one block per row and instance)
// listed instances k = blockIdx.y, blockIdx.y + gridDim.y, ... < nmax (a
// negative list entry ends the list)
// DF: the result as a float-float pair (the GMRES path's operand) in the same
// 8 bytes per entry, else FP64 (the FP64 Newton matrix path)
template <bool DF>
__global__ void k_rom_gu64(RomDev d, const double* __restrict__ G, const int* __restrict__ active,
                           const int* __restrict__ hp, const int* __restrict__ hplist, int nmax,
                           double* __restrict__ GU) {
    const int p = blockIdx.x;
    const int32_t* gi = d.gidx + (int64_t)p * GMAX;
    for (int k = blockIdx.y; k < nmax; k += gridDim.y) {
        const int b = hplist[k];
        if (b < 0) return;
        if (!active[b] || !hp[b]) continue;
        const double* Gp = G + ((int64_t)b * d.M + p) * GMAX;
        for (int j = threadIdx.x; j < d.Nr; j += blockDim.x) {
            double acc = 0.0;
            for (int e = 0; e < GMAX; ++e) {
                const int s = gi[e];
                if (s < 0) break;
                acc += Gp[e] * d.UlocR[(int64_t)s * d.Nr + j];
            }
            const int64_t o = ((int64_t)b * d.M + p) * d.Nr + j;
            if (DF) reinterpret_cast<float2*>(GU)[o] = df_from_double(acc);
            else GU[o] = acc;
        }
    }
}
__global__ void k_rom_jac64(RomDev d, const double* __restrict__ prm, const double* __restrict__ GU,
                            const int* __restrict__ active, const int* __restrict__ hp,
                            const int* __restrict__ hplist, int nmax, double* __restrict__ J) {
    const int i = blockIdx.x;
    const double* Pi = d.P + (int64_t)i * d.M;
    for (int k = blockIdx.y; k < nmax; k += gridDim.y) {
        const int b = hplist[k];
        if (b < 0) return;
        if (!active[b] || !hp[b]) continue;
        const double dt_inv = prm[RP * b + 3];
        const double* GUb = GU + (int64_t)b * d.M * d.Nr;
        for (int j = threadIdx.x; j < d.Nr; j += blockDim.x) {
            double acc = d.Ms[(int64_t)i * d.Nr + j] * dt_inv + d.Alin[(int64_t)i * d.Nr + j];
            for (int p = 0; p < d.M; ++p) acc += Pi[p] * GUb[(int64_t)p * d.Nr + j];
            J[((int64_t)b * d.Nr + i) * d.Nr + j] = acc;
        }
    }
}

// r[b] = Ms (a - a_old)/dt + Alin a + mu bbnd + P f[b] (FP64); one block per
// instance, one warp per row, lanes over the columns, a fixed shuffle tree
__global__ void __launch_bounds__(256)
k_rom_resid(RomDev d, const double* __restrict__ a, const double* __restrict__ a_old,
            const double* __restrict__ prm, const double* __restrict__ f, const int* __restrict__ active,
            double* __restrict__ r) {
    const int b = blockIdx.x;
    if (!active[b]) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double dt_inv = prm[RP * b + 3];
    const double* ab = a + (int64_t)b * d.Nr;
    const double* aob = a_old + (int64_t)b * d.Nr;
    const double* fb = f + (int64_t)b * d.M;
    const double mu = prm[RP * b];
    for (int i = wid; i < d.Nr; i += nw) {
        double acc = 0.0;
        for (int j = lane; j < d.Nr; j += 32)
            acc += d.Ms[(int64_t)i * d.Nr + j] * (ab[j] - aob[j]) * dt_inv + d.Alin[(int64_t)i * d.Nr + j] * ab[j];
        for (int p = lane; p < d.M; p += 32) acc += d.P[(int64_t)i * d.M + p] * fb[p];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) r[(int64_t)b * d.Nr + i] = acc + mu * d.bbnd[i];
    }
}

// delta[b] = -J[b]^-1 r[b] in the precision T of J (r and delta FP64): row
// then column equilibration, LU with partial pivoting (ties: lowest row),
// forward elimination of the right-hand side during the factorisation (so the
// L factor is stored only with KEEP), back substitution.  One block per instance; the
// matrix is copied to shared memory (SMEM, lu_smem(Nr, sizeof(T)) <=
// ROM_LU_SMEM, opt-in above 48 KB, set at mb_rom_create), or, when it does not
// fit, its leading rows as far as the dynamic shared memory reaches, the other
// rows factorised in place in J (row swaps move data between the two).  Per column k: warp 0 reduces the per-warp pivot candidates, all threads
// swap the two rows, then warp w eliminates rows k+1+w, k+1+w+nw, ... with its
// lanes along the columns and keeps the largest |A[i][k+1]| of its rows as the
// next column's candidate (two or three barriers per column).  1/A[k][k] is
// kept in x[k] for warp 0's back substitution.  128 threads up to Nr 96, 1024
// beyond (one block per SM at the larger sizes: warps hide the latency).
// KEEP: the factors stay in J (whole rows swapped, multipliers stored below
// the diagonal), with the pivot rows in piv_out[b] and the row and column
// scales in sc_out[b] (Nr each), for k_rom_gmres's preconditioner.
constexpr int ROM_LU_SMEM = 220 * 1024;
constexpr int LU_T_SMALL = 128, LU_T_LARGE = 1024;
__host__ __device__ constexpr size_t lu_smem(int Nr, size_t elem) { return elem * ((size_t)Nr * Nr + 4 * (size_t)Nr); }
template <class T>
__device__ inline void lu_pick(T& best, int& bi, T v2, int i2) {
    if (v2 > best || (v2 == best && i2 < bi)) { best = v2; bi = i2; }
}
template <class T, bool SMEM, bool KEEP = false>
__global__ void __launch_bounds__(1024, 1)
k_rom_lu(int Nr, T* __restrict__ J, const double* __restrict__ r, const int* __restrict__ active,
         const int* __restrict__ hp, int want_hp, const int* __restrict__ list, double* __restrict__ delta,
         int* __restrict__ piv_out = nullptr, T* __restrict__ sc_out = nullptr) {
    const int b = list ? list[blockIdx.x] : blockIdx.x;
    if (b < 0) return;   // past the end of the list (launched for the whole batch)
    if (!active[b] || (hp[b] != 0) != (want_hp != 0)) return;
    extern __shared__ __align__(16) unsigned char lu_raw[];
    T* const sm = reinterpret_cast<T*>(lu_raw);
    T* const Jb = J + (int64_t)b * Nr * Nr;
    T* const rs = sm;                            // row scales
    T* const cs = rs + Nr;                       // column scales
    T* const rhs = cs + Nr;
    T* const x = rhs + Nr;                       // 1/A[k][k], then the solution
    T* const rows = x + Nr;                      // rows [0, R) of the matrix in shared memory
    // rows that fit in the dynamic shared memory (all with SMEM); the others
    // are factorised in place in J
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const int R = SMEM ? Nr : min(Nr, max(0, (int)(dyn / sizeof(T)) - 4 * Nr) / Nr);
    auto row = [&](int i) -> T* { return i < R ? rows + (size_t)i * Nr : Jb + (size_t)i * Nr; };
    __shared__ T wbest[32];
    __shared__ int widx[32];
    __shared__ int spiv;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int e = tid; e < R * Nr; e += blockDim.x) rows[e] = Jb[e];
    __syncthreads();
    for (int i = wid; i < Nr; i += nw) {
        const T* ri = row(i);
        T m = T(0);
        for (int j = lane; j < Nr; j += 32) m = fmax(m, fabs(ri[j]));
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) rs[i] = m > T(0) ? T(1) / m : T(1);
    }
    __syncthreads();
    for (int j = tid; j < Nr; j += blockDim.x) {
        T m = T(0);
        for (int i = 0; i < Nr; ++i) m = fmax(m, fabs(row(i)[j] * rs[i]));
        cs[j] = m > T(0) ? T(1) / m : T(1);
    }
    __syncthreads();
    for (int i = wid; i < Nr; i += nw) {
        T* ri = row(i);
        for (int j = lane; j < Nr; j += 32) ri[j] *= rs[i] * cs[j];
    }
    for (int i = tid; i < Nr; i += blockDim.x) rhs[i] = (T)(-r[(int64_t)b * Nr + i]) * rs[i];
    __syncthreads();
    {
        // candidates for the first pivot
        T best = T(-1);
        int bi = Nr;
        for (int i = tid; i < Nr; i += blockDim.x) lu_pick(best, bi, fabs(row(i)[0]), i);
        for (int o = 16; o > 0; o >>= 1)
            lu_pick(best, bi, __shfl_xor_sync(0xffffffffu, best, o), __shfl_xor_sync(0xffffffffu, bi, o));
        if (lane == 0) {
            wbest[wid] = best;
            widx[wid] = bi;
        }
    }
    __syncthreads();
    for (int k = 0; k < Nr; ++k) {
        if (wid == 0) {
            T best = lane < nw ? wbest[lane] : T(-1);
            int bi = lane < nw ? widx[lane] : Nr;
            for (int o = 16; o > 0; o >>= 1)
                lu_pick(best, bi, __shfl_xor_sync(0xffffffffu, best, o), __shfl_xor_sync(0xffffffffu, bi, o));
            if (lane == 0) spiv = bi < Nr ? bi : k;
        }
        __syncthreads();
        const int piv = spiv;   // the same in every thread: the branch below is uniform
        if (KEEP && tid == 0) piv_out[(int64_t)b * Nr + k] = piv;
        T* const rk = row(k);
        if (piv != k) {
            T* const rp = row(piv);
            for (int j = (KEEP ? 0 : k) + tid; j < Nr; j += blockDim.x) {
                const T t = rk[j];
                rk[j] = rp[j];
                rp[j] = t;
            }
            if (tid == 0) {
                const T t = rhs[k];
                rhs[k] = rhs[piv];
                rhs[piv] = t;
            }
            __syncthreads();
        }
        const T akk = rk[k];
        const T inv = akk != T(0) ? T(1) / akk : T(0);
        const T rkk = rhs[k];
        if (tid == 0) x[k] = inv;
        T best = T(-1);
        int bi = Nr;
        // row i minus l times the pivot row; the callers below pass pointers whose
        // memory (shared or global) the compiler sees, so that shared-memory rows
        // are accessed with shared-memory instructions rather than generic ones
        auto elim = [&](T* ri, const T* rkp, int i) {
            const T l = ri[k] * inv;
            int j = k + 1 + lane;
            if (j < Nr) {   // column k+1 (lane 0) feeds the next pivot search
                const T v = ri[j] - l * rkp[j];
                ri[j] = v;
                if (lane == 0) lu_pick(best, bi, fabs(v), i);
                j += 32;
            }
#pragma unroll 4
            for (; j < Nr; j += 32) ri[j] -= l * rkp[j];
            if (KEEP) {
                __syncwarp();   // every lane has read A[i][k] before lane 0 overwrites it
                if (lane == 0) ri[k] = l;
            }
            if (lane == 0) rhs[i] -= l * rkk;
        };
        auto sweep = [&](const T* rkp) {
            for (int i = k + 1 + wid; i < Nr; i += nw) {
                if (SMEM || i < R) elim(rows + (size_t)i * Nr, rkp, i);
                else elim(Jb + (size_t)i * Nr, rkp, i);
            }
        };
        if (SMEM || k < R) sweep(rows + (size_t)k * Nr);
        else sweep(Jb + (size_t)k * Nr);
        if (lane == 0) {   // column k+1 lives in lane 0 of every warp
            wbest[wid] = best;
            widx[wid] = bi;
        }
        __syncthreads();
    }
    if (wid == 0) {
        for (int k = Nr - 1; k >= 0; --k) {
            const T* rk = row(k);
            T part = T(0);
            for (int j = k + 1 + lane; j < Nr; j += 32) part += rk[j] * x[j];
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) x[k] = (rhs[k] - part) * x[k];
            __syncwarp();
        }
    }
    __syncthreads();
    for (int j = tid; j < Nr; j += blockDim.x) delta[(int64_t)b * Nr + j] = (double)(x[j] * cs[j]);
    if (KEEP) {
        for (int e = tid; e < R * Nr; e += blockDim.x) Jb[e] = rows[e];
        for (int j = tid; j < Nr; j += blockDim.x) {
            sc_out[(int64_t)b * 2 * Nr + j] = rs[j];
            sc_out[(int64_t)b * 2 * Nr + Nr + j] = cs[j];
        }
    }
}

// Launch the LU solve of the listed instances (all B without a list) with
// want_hp selecting the FP32 (0) or FP64 (1) Newton matrices.
template <class T>
static void launch_rom_lu(int Nr, int nblk, T* J, const double* r, const int* active, const int* hp, int want_hp,
                          const int* list, double* delta, cudaStream_t s, int* piv = nullptr, T* sc = nullptr) {
    const unsigned lt = Nr <= 96 ? LU_T_SMALL : LU_T_LARGE;
    if (piv) {   // keep the factors
        if (lu_smem(Nr, sizeof(T)) <= ROM_LU_SMEM)
            k_rom_lu<T, true, true><<<(unsigned)nblk, lt, lu_smem(Nr, sizeof(T)), s>>>(Nr, J, r, active, hp, want_hp,
                                                                                       list, delta, piv, sc);
        else
            k_rom_lu<T, false, true><<<(unsigned)nblk, lt, ROM_LU_SMEM, s>>>(
                Nr, J, r, active, hp, want_hp, list, delta, piv, sc);
        return;
    }
    if (lu_smem(Nr, sizeof(T)) <= ROM_LU_SMEM)
        k_rom_lu<T, true><<<(unsigned)nblk, lt, lu_smem(Nr, sizeof(T)), s>>>(Nr, J, r, active, hp, want_hp, list,
                                                                             delta);
    else
        k_rom_lu<T, false><<<(unsigned)nblk, lt, ROM_LU_SMEM, s>>>(Nr, J, r, active, hp, want_hp, list, delta);
}

// Newton step of an escalated instance (hp[b], refinement mode): delta =
// -J64^-1 r by right-preconditioned restarted GMRES(m) in FP64 on products
// J64 z = Ms z/dt + Alin z + P (GU64[b] z) (GU64 = G U_loc in FP64, formed by
// k_rom_gu64; the FP64 Newton matrix itself is never formed), preconditioned by
// the instance's FP32 LU kept from its last FP32-matrix iteration (row scales,
// row swaps, unit-lower and upper triangular solves, column scales; FP64
// arithmetic on the FP32 factors).  Stops when the residual estimate falls
// below eta |r| or after `cycles` restarts; Arnoldi by classical Gram-Schmidt
// with one reorthogonalisation, Givens rotations on thread 0.  One block of
// 256 threads per listed instance; shared memory gmres_smem(Nr, M, m) doubles.
__host__ __device__ constexpr size_t gmres_smem(int Nr, int M, int m) {
    return 8 * ((size_t)(m + 1) * Nr + (size_t)M + 4 * (size_t)Nr + (size_t)(m + 1) * m + 4 * (size_t)(m + 1) + 40 +
                ((size_t)Nr + 1) / 2);
}
constexpr int GMRES_M = 16, GMRES_CYCLES = 2;
constexpr double GMRES_ETA = 1e-6;
__device__ inline double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__global__ void __launch_bounds__(256)
k_rom_gmres(RomDev d, const double* __restrict__ prm, const double* __restrict__ GU64, const double* __restrict__ r,
            const float* __restrict__ J, const int* __restrict__ lpiv, const float* __restrict__ lsc,
            const int* __restrict__ active, const int* __restrict__ hp, const int* __restrict__ hplist, int m,
            int cycles, double eta, double* __restrict__ delta) {
    const int b = hplist[blockIdx.x];
    if (b < 0) return;   // past the end of the list (launched for the whole batch)
    if (!active[b] || !hp[b]) return;
    const int Nr = d.Nr, M = d.M;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    extern __shared__ __align__(16) unsigned char gm_raw[];
    double* const V = reinterpret_cast<double*>(gm_raw);   // (m+1) x Nr Krylov basis
    double* const t = V + (size_t)(m + 1) * Nr;           // M: GU64 z
    double* const z = t + M;                              // Nr
    double* const w = z + Nr;                             // Nr
    double* const x = w + Nr;                             // Nr: the solution
    double* const H = x + Nr;                             // (m+1) x m, column j at H + j (m+1)
    double* const gv = H + (size_t)(m + 1) * m;           // m+1: rotated right-hand side
    double* const cr = gv + (m + 1);                      // m: Givens cosines
    double* const sr = cr + (m + 1);                      // m: Givens sines
    double* const hy = sr + (m + 1);                      // m+1: projections, then y
    float2* const sdf = reinterpret_cast<float2*>(hy + (m + 1));   // Nr: the product's input as float-float
    double* const red = hy + (m + 1) + Nr;                // 40: reduction scratch and flags
    int* const ps = reinterpret_cast<int*>(red + 40);     // Nr pivot rows
    const float* const LU = J + (int64_t)b * Nr * Nr;
    const int* const pv = lpiv + (int64_t)b * Nr;
    const float* const rsc = lsc + (int64_t)b * 2 * Nr;
    const float* const csc = rsc + Nr;
    // the instance's G U_loc as float-float pairs (k_rom_gu64<true>)
    const float2* const GUb = reinterpret_cast<const float2*>(GU64) + (int64_t)b * M * Nr;
    float2* const tdf = reinterpret_cast<float2*>(t);
    const double dt_inv = prm[RP * b + 3];
    for (int k = tid; k < Nr; k += blockDim.x) ps[k] = pv[k];

    // sum over the block of one value per thread, returned to every thread
    auto block_sum = [&](double v) -> double {
        v = warp_sum_d(v);
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (wid == 0) {
            double u = lane < nw ? red[lane] : 0.0;
            u = warp_sum_d(u);
            if (lane == 0) red[32] = u;
        }
        __syncthreads();
        const double tot = red[32];
        __syncthreads();
        return tot;
    };
    // dst = M^-1 src (src, dst distinct shared vectors): the instance's FP32 LU
    // applied in FP32 (a fixed linear operator up to rounding; only GMRES's
    // convergence depends on it, the products and the residual set the
    // step's accuracy), row-oriented triangular solves on warp 0
    float* const yf = reinterpret_cast<float*>(sdf);   // Nr floats (sdf is free outside the products)
    auto precond = [&](const double* src, double* dst) {
        for (int i = tid; i < Nr; i += blockDim.x) yf[i] = (float)((double)rsc[i] * src[i]);
        __syncthreads();
        if (tid == 0)
            for (int k = 0; k < Nr; ++k) {
                const int p = ps[k];
                if (p != k) {
                    const float tmp = yf[k];
                    yf[k] = yf[p];
                    yf[p] = tmp;
                }
            }
        __syncthreads();
        if (wid == 0) {
            for (int i = 1; i < Nr; ++i) {   // unit lower triangle
                float a = 0.f;
                const float* Li = LU + (int64_t)i * Nr;
                for (int k = lane; k < i; k += 32) a = fmaf(Li[k], yf[k], a);
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) yf[i] -= a;
                __syncwarp();
            }
            for (int i = Nr - 1; i >= 0; --i) {   // upper triangle
                float a = 0.f;
                const float* Ui = LU + (int64_t)i * Nr;
                for (int k = i + 1 + lane; k < Nr; k += 32) a = fmaf(Ui[k], yf[k], a);
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) {
                    const float u = Ui[i];
                    yf[i] = u != 0.f ? (yf[i] - a) / u : 0.f;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int i = tid; i < Nr; i += blockDim.x) dst[i] = (double)yf[i] * (double)csc[i];
        __syncthreads();
    };
    // dst = J src with J = Ms/dt + Alin + P (G U_loc): float-float operands and
    // compensated dot products (Dot2 of Ogita, Rump and Oishi, "Accurate sum
    // and dot product", SIAM J. Sci. Comput. 26, 2005: TwoProduct per term,
    // TwoSum into the running sum, the errors gathered in a second FP32 sum),
    // as accurate as a dot product in ~48-bit arithmetic, on the FP32 pipe
    // (GB300's FP64 pipe took ~64x longer for these products)
    auto dot2 = [](float2 a, float2 b, float& sh, float& sc) {
        const float pr = a.x * b.x;
        float q = fmaf(a.x, b.x, -pr);
        q = fmaf(a.x, b.y, fmaf(a.y, b.x, q));
        const float tt = sh + pr, z = tt - sh;
        sc += q + ((sh - (tt - z)) + (pr - z));
        sh = tt;
    };
    auto dot2_warp = [](float& sh, float& sc) {
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_xor_sync(0xffffffffu, sh, o), c2 = __shfl_xor_sync(0xffffffffu, sc, o);
            const float tt = sh + s2, z = tt - sh;
            sc += c2 + ((sh - (tt - z)) + (s2 - z));
            sh = tt;
        }
    };
    auto matvec = [&](const double* src, double* dst) {
        for (int j = tid; j < Nr; j += blockDim.x) sdf[j] = df_from_double(src[j]);
        __syncthreads();
        for (int p = wid; p < M; p += nw) {
            float sh = 0.f, sc = 0.f;
            for (int j = lane; j < Nr; j += 32) dot2(GUb[(int64_t)p * Nr + j], sdf[j], sh, sc);
            dot2_warp(sh, sc);
            if (lane == 0) tdf[p] = df_fast2sum(sh, sc);
        }
        __syncthreads();
        for (int i = wid; i < Nr; i += nw) {
            float s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f, s3 = 0.f, c3 = 0.f;
            for (int p = lane; p < M; p += 32) dot2(d.Pdf[(int64_t)i * M + p], tdf[p], s1, c1);
            for (int j = lane; j < Nr; j += 32) {
                dot2(d.Msdf[(int64_t)i * Nr + j], sdf[j], s2, c2);
                dot2(d.Alindf[(int64_t)i * Nr + j], sdf[j], s3, c3);
            }
            dot2_warp(s1, c1);
            dot2_warp(s2, c2);
            dot2_warp(s3, c3);
            if (lane == 0)
                dst[i] = ((double)s1 + (double)c1) + dt_inv * ((double)s2 + (double)c2) + ((double)s3 + (double)c3);
        }
        __syncthreads();
    };

    for (int i = tid; i < Nr; i += blockDim.x) x[i] = 0.0;
    __syncthreads();
    double beta0 = 0.0;
    for (int cyc = 0; cyc < cycles; ++cyc) {
        // w = -r - J64 x
        if (cyc == 0) {
            for (int i = tid; i < Nr; i += blockDim.x) w[i] = -r[(int64_t)b * Nr + i];
            __syncthreads();
        } else {
            matvec(x, w);
            for (int i = tid; i < Nr; i += blockDim.x) w[i] = -r[(int64_t)b * Nr + i] - w[i];
            __syncthreads();
        }
        double ss = 0.0;
        for (int i = tid; i < Nr; i += blockDim.x) ss += w[i] * w[i];
        const double beta = sqrt(block_sum(ss));
        if (cyc == 0) beta0 = beta;
        if (!(beta > eta * beta0) || !(beta > 0.0)) break;   // converged, zero or not finite
        for (int i = tid; i < Nr; i += blockDim.x) V[i] = w[i] / beta;
        if (tid == 0) {
            gv[0] = beta;
            for (int i = 1; i <= m; ++i) gv[i] = 0.0;
        }
        __syncthreads();
        int kdim = 0;
        for (int j = 0; j < m; ++j) {
            precond(V + (size_t)j * Nr, z);
            matvec(z, w);
            double* const Hj = H + (size_t)j * (m + 1);
            for (int pass = 0; pass < 2; ++pass) {
                for (int i = wid; i <= j; i += nw) {
                    double a = 0.0;
                    for (int l = lane; l < Nr; l += 32) a += V[(size_t)i * Nr + l] * w[l];
                    a = warp_sum_d(a);
                    if (lane == 0) hy[i] = a;
                }
                __syncthreads();
                for (int l = tid; l < Nr; l += blockDim.x) {
                    double a = w[l];
                    for (int i = 0; i <= j; ++i) a -= hy[i] * V[(size_t)i * Nr + l];
                    w[l] = a;
                }
                if (tid == 0)
                    for (int i = 0; i <= j; ++i) Hj[i] = (pass ? Hj[i] : 0.0) + hy[i];
                __syncthreads();
            }
            double sw = 0.0;
            for (int l = tid; l < Nr; l += blockDim.x) sw += w[l] * w[l];
            const double hn = sqrt(block_sum(sw));
            for (int l = tid; l < Nr; l += blockDim.x) V[(size_t)(j + 1) * Nr + l] = hn > 0.0 ? w[l] / hn : 0.0;
            if (tid == 0) {
                Hj[j + 1] = hn;
                for (int i = 0; i < j; ++i) {   // earlier rotations
                    const double h0 = Hj[i], h1 = Hj[i + 1];
                    Hj[i] = cr[i] * h0 + sr[i] * h1;
                    Hj[i + 1] = -sr[i] * h0 + cr[i] * h1;
                }
                const double a0 = Hj[j], a1 = Hj[j + 1];
                const double rho = hypot(a0, a1);
                const double c = rho > 0.0 ? a0 / rho : 1.0, sn = rho > 0.0 ? a1 / rho : 0.0;
                cr[j] = c;
                sr[j] = sn;
                Hj[j] = rho;
                Hj[j + 1] = 0.0;
                gv[j + 1] = -sn * gv[j];
                gv[j] = c * gv[j];
                red[33] = (!(fabs(gv[j + 1]) > eta * beta0) || !(hn > 0.0)) ? 1.0 : 0.0;
            }
            __syncthreads();
            kdim = j + 1;
            const bool done = red[33] != 0.0;
            __syncthreads();
            if (done) break;
        }
        // y = H^-1 g (upper triangular, kdim x kdim); x += M^-1 (V y)
        if (tid == 0)
            for (int i = kdim - 1; i >= 0; --i) {
                double a = gv[i];
                for (int l = i + 1; l < kdim; ++l) a -= H[(size_t)l * (m + 1) + i] * hy[l];
                const double hii = H[(size_t)i * (m + 1) + i];
                hy[i] = hii != 0.0 ? a / hii : 0.0;
            }
        __syncthreads();
        for (int l = tid; l < Nr; l += blockDim.x) {
            double a = 0.0;
            for (int i = 0; i < kdim; ++i) a += hy[i] * V[(size_t)i * Nr + l];
            w[l] = a;
        }
        __syncthreads();
        precond(w, z);
        for (int l = tid; l < Nr; l += blockDim.x) x[l] += z[l];
        __syncthreads();
    }
    // a residual that is not finite gives a step that is not, as the LU path does
    for (int l = tid; l < Nr; l += blockDim.x) delta[(int64_t)b * Nr + l] = isfinite(beta0) ? x[l] : beta0;
}

// Step length of all instances: the scaled max-norm of the reconstructed
// update U_loc delta over the closure (FP32; it only sets the step length
// and the stop), as a tiled product U_loc [delta_0 | delta_1 | ...]: a block
// takes UN_K closure slots x UN_B instances, K (the reduced coordinates) in
// chunks of 16 staged in shared memory, each thread 4 x 4 results; per
// instance and tile the maximum goes to dpart (NaN counts as infinite).
constexpr int UN_K = 128, UN_B = 32, UN_C = 16;
__global__ void __launch_bounds__(256)
k_rom_unorm(RomDev d, int B, const double* __restrict__ delta, const int* __restrict__ active,
            const double* __restrict__ uloc, float* __restrict__ dpart) {
    __shared__ float Us[UN_C][UN_K];
    __shared__ float Ds[UN_C][UN_B];
    const int k0 = blockIdx.x * UN_K, b0 = blockIdx.y * UN_B;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 slot groups x 8 instance groups
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[u][q] = 0.f;
    for (int j0 = 0; j0 < d.Nr; j0 += UN_C) {
        for (int e = threadIdx.x; e < UN_C * UN_K; e += 256) {
            const int j = e / UN_K, k = e % UN_K;
            Us[j][k] = (j0 + j < d.Nr && k0 + k < d.nloc) ? d.UlocCf[(int64_t)(j0 + j) * d.nloc + k0 + k] : 0.f;
        }
        for (int e = threadIdx.x; e < UN_C * UN_B; e += 256) {
            const int j = e / UN_B, q = e % UN_B;
            const int b = b0 + q;
            Ds[j][q] = (j0 + j < d.Nr && b < B) ? (float)delta[(int64_t)b * d.Nr + j0 + j] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < UN_C; ++j) {
            float u[4], v[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) u[s] = Us[j][tx + 32 * s];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = Ds[j][ty * 4 + q];
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[s][q] = fmaf(u[s], v[q], acc[s][q]);
        }
        __syncthreads();
    }
    // per instance: max over this thread's 4 slots, then over the warp's 32
    // threads: over every slot in the unknown scales (dpart) and for the
    // step-length cap (dpart + B * gridDim.x: voxel slots in their scales,
    // face slots relative to max(n_c, |n|) of the current reconstruction)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float m = 0.f, mc = 0.f;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int k = k0 + tx + 32 * s;
            const int bq = b0 + ty * 4 + q;
            if (k < d.nloc && bq < B) {
                const float a = fabsf(acc[s][q]);
                const float sc = d.uscf[k];
                const float v = a / d.usf[k];
                const float vc = sc > 0.f ? a / sc : a / fmaxf(d.ncf, fabsf((float)uloc[(int64_t)bq * d.nloc + k]));
                m = (v == v) ? fmaxf(m, v) : INFINITY;
                mc = (vc == vc) ? fmaxf(mc, vc) : INFINITY;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            mc = fmaxf(mc, __shfl_xor_sync(0xffffffffu, mc, o));
        }
        const int b = b0 + ty * 4 + q;
        if (tx == 0 && b < B) {
            dpart[(int64_t)b * gridDim.x + blockIdx.x] = m;
            dpart[((int64_t)B + b) * gridDim.x + blockIdx.x] = mc;
        }
    }
}

// step length and convergence of instance b from the partial maxima (one warp per instance)
__global__ void __launch_bounds__(32)
k_rom_apply(RomDev d, int B, int nkt, double* __restrict__ a, const double* __restrict__ delta,
            const float* __restrict__ dpart, int* __restrict__ active, int* __restrict__ failed,
            long long* __restrict__ its, int* __restrict__ pit, int* __restrict__ hp, float* __restrict__ dnprev,
            int rate) {
    const int b = blockIdx.x, lane = threadIdx.x;
    if (!active[b]) return;
    float m = 0.f, mc = 0.f;
    for (int t = lane; t < nkt; t += 32) {
        const float v = dpart[(int64_t)b * nkt + t], vc = dpart[((int64_t)B + b) * nkt + t];
        m = (v == v) ? fmaxf(m, v) : INFINITY;
        mc = (vc == vc) ? fmaxf(mc, vc) : INFINITY;
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        mc = fmaxf(mc, __shfl_xor_sync(0xffffffffu, mc, o));
    }
    const double dn = (double)m, dv = (double)mc;
    if (!(dn < INFINITY)) {
        if (lane == 0) { failed[b] = 2; active[b] = 0; }   // 2: a non-finite update
        return;
    }
    // step length and convergence in the same scaled max-norm: voxel slots in
    // their scales, plated inventories relative to max(n_c, |n|) (in units of
    // n_c alone, the rounding of a thick stripping layer's reconstruction,
    // amplified by the exponential kinetics, stays above the tolerance)
    const double lam = dv <= ROM_DELTA_MAX ? 1.0 : ROM_DELTA_MAX / dv;
    for (int j = lane; j < d.Nr; j += 32) a[(int64_t)b * d.Nr + j] += lam * delta[(int64_t)b * d.Nr + j];
    if (lane == 0) {
        its[b] += 1;
        const int k = ++pit[b];
        // converged: below the tolerance, or a full step below ROM_TOL_FLOOR that no
        // longer halves the previous update (the iteration has reached the rounding
        // floor of the reconstruction; Newton's own convergence is quadratic), or
        // (rate) a full step after a full step whose estimated remaining error
        // rho / (1 - rho) dv, rho = dv / dv_prev < 0.5, is below the tolerance
        const double dvp = (double)dnprev[b];
        const bool by_rate = rate && lam == 1.0 && k >= 2 && dvp <= ROM_DELTA_MAX && dv < 0.5 * dvp &&
                             dv / (dvp - dv) * dv <= ROM_TOL;
        if (lam * dv <= ROM_TOL || (lam == 1.0 && dv <= ROM_TOL_FLOOR && k >= 2 && mc >= 0.5f * dnprev[b]) || by_rate)
            active[b] = 0;
        if (k >= ROM_HP_AFTER || (k >= 3 && lam == 1.0 && mc > 0.9f * dnprev[b])) hp[b] = 1;
        dnprev[b] = mc;
    }
}

// out[0] = active instances, out[1] = escalated (FP64) instances
// (active or not), listed in list[0, out[1]) (one block; the list's order
// does not matter: every instance's arithmetic is its own)
// out[2] = active instances on the FP32 matrix, listed in alist[0, out[2])
__global__ void k_rom_count_hp(int B, const int* __restrict__ active, const int* __restrict__ hp,
                               int* __restrict__ out, int* __restrict__ list, int* __restrict__ alist) {
    __shared__ int c0, c1, c2;
    if (threadIdx.x == 0) { c0 = 0; c1 = 0; c2 = 0; }
    __syncthreads();
    int a = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        a += active[b] != 0;
        if (hp[b]) list[atomicAdd(&c1, 1)] = b;
        else if (active[b]) alist[atomicAdd(&c2, 1)] = b;
    }
    atomicAdd(&c0, a);
    __syncthreads();
    if (threadIdx.x == 0) { out[0] = c0; out[1] = c1; out[2] = c2; }
    // end both lists with -1 (kernels launched for the whole batch stop there)
    for (int b = c1 + threadIdx.x; b < B; b += blockDim.x) list[b] = -1;
    for (int b = c2 + threadIdx.x; b < B; b += blockDim.x) alist[b] = -1;
}

// copy src -> dst for instances with mask[b] (all instances if mask is null)
__global__ void k_rom_copy(int Nr, int B, const int* __restrict__ mask, const double* __restrict__ src,
                           double* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * Nr) return;
    if (mask && !mask[i / Nr]) return;
    dst[i] = src[i];
}

// active = on && !failed; pit (if given) = 0; hp (if given) = 0
__global__ void k_rom_set_active(int B, const int* __restrict__ on, const int* __restrict__ failed,
                                 int* __restrict__ active, int* __restrict__ pit, int* __restrict__ hp) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    active[b] = (on ? on[b] : 1) && !failed[b];
    if (pit) pit[b] = 0;
    if (hp) hp[b] = 0;
}

// flips of pass-active instances; instances with flips stay on for the next pass
// (g1 and gate may be the same buffer: g1 is read before the barrier, gate written after it)
__global__ void k_rom_flips(int ngate, int B, const uint8_t* g1, const uint8_t* __restrict__ g2,
                            const int* __restrict__ failed, int* __restrict__ pass_on, long long* __restrict__ flips,
                            uint8_t* gate, int last_pass, const int* __restrict__ dpass) {
    if (dpass) last_pass = *dpass + 1 >= ROM_PASSES;   // pass number kept on the device (graph launch)
    const int b = blockIdx.x;
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    if (!pass_on[b] || failed[b]) {
        if (threadIdx.x == 0) pass_on[b] = 0;
        return;
    }
    int c = 0;
    for (int g = threadIdx.x; g < ngate; g += blockDim.x)
        c += g1[(int64_t)b * ngate + g] != g2[(int64_t)b * ngate + g];
    atomicAdd(&cnt, c);
    __syncthreads();
    if (cnt > 0 && !last_pass) {
        for (int g = threadIdx.x; g < ngate; g += blockDim.x) gate[(int64_t)b * ngate + g] = g2[(int64_t)b * ngate + g];
    }
    if (threadIdx.x == 0) {
        if (cnt > 0 && !last_pass) flips[b] += cnt;
        pass_on[b] = (cnt > 0 && !last_pass) ? 1 : 0;
    }
}

__global__ void k_rom_outputs(RomDev d, int B, const double* __restrict__ a, double* __restrict__ V,
                              double* __restrict__ S) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double v = 0.0, s = 0.0;
    for (int j = 0; j < d.Nr; ++j) {
        v += d.scp[j] * a[(int64_t)b * d.Nr + j];
        s += d.sac[j] * a[(int64_t)b * d.Nr + j];
    }
    V[b] = v;
    S[b] = s;
}

// start slot b: a = a0, parameters, counters zero, not failed
__global__ void k_rom_slot_start(RomDev d, int b, double I_app, double s_i0, double k_pl, double dt_inv,
                                 double* __restrict__ a, double* __restrict__ prm, int* __restrict__ failed,
                                 long long* __restrict__ its, long long* __restrict__ flips, int* __restrict__ hp) {
    for (int j = threadIdx.x; j < d.Nr; j += blockDim.x) a[(int64_t)b * d.Nr + j] = d.a0[j];
    if (threadIdx.x == 0) {
        prm[RP * b] = I_app;
        prm[RP * b + 1] = s_i0;
        prm[RP * b + 2] = k_pl;
        prm[RP * b + 3] = dt_inv;
        failed[b] = 0;
        its[b] = 0;
        flips[b] = 0;
        hp[b] = 0;
    }
}

// start every slot b < B (parameters already in prm): a = a0, counters zero, not failed
__global__ void k_rom_batch_start(RomDev d, int B, double* __restrict__ a, int* __restrict__ failed,
                                  long long* __restrict__ its, long long* __restrict__ flips, int* __restrict__ hp) {
    const int64_t n = (int64_t)B * d.Nr;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / d.Nr), j = (int)(e - (int64_t)b * d.Nr);
        a[e] = d.a0[j];
        if (j == 0) {
            failed[b] = 0;
            its[b] = 0;
            flips[b] = 0;
            hp[b] = 0;
        }
    }
}

__global__ void k_rom_fail_active(int B, int* __restrict__ active, int* __restrict__ failed) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B && active[b]) {
        failed[b] = 1;   // 1: still iterating after the iteration limit
        active[b] = 0;
    }
}

__global__ void k_rom_count(int B, const int* __restrict__ flag, int* __restrict__ out) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) c += flag[b] != 0;
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) *out = cnt;
}

// ------------------------------------------------------------- host build
namespace {

struct HostCell {
    int nt, ny, nz;
    int64_t N, F, syz;
    std::vector<uint32_t> vc;
    std::vector<int32_t> pg, pe;
    int phase(int64_t v) const { return (int)(vc[v] & 7u); }
    int64_t nb(int64_t v, int d) const {
        int z = (int)(v % nz), y = (int)((v / nz) % ny), t = (int)(v / syz);
        switch (d) {
            case 0: return t > 0 ? v - syz : -1;
            case 1: return t < nt - 1 ? v + syz : -1;
            case 2: return y > 0 ? v - nz : -1;
            case 3: return y < ny - 1 ? v + nz : -1;
            case 4: return z > 0 ? v - 1 : -1;
            default: return z < nz - 1 ? v + 1 : -1;
        }
    }
    // interface face of solid s towards direction d
    int64_t iface(int64_t s, int d) const {
        uint32_t c = vc[s];
        uint32_t m = (c >> 3) & 63u;
        return (int64_t)(c >> VC_FBASE_SHIFT) + __builtin_popcount(m & ((1u << d) - 1u));
    }
};

bool kinetic(int p) { return p == PG || p == PK || p == PL; }

struct Term {
    int type = T_NONE;
    int64_t dof[5] = {-1, -1, -1, -1, -1};   // full-state indices
    double wbv = 0.0, wpl = 0.0;
    int64_t face = -1;                        // plating face (gate)
};

}  // namespace

static int rom_build_host(mb_rom* R, const mb_rom_data* dd) {
    mb_cell* c = R->cell;
    const Dims& D = c->D;
    HostCell H;
    H.nt = D.nt; H.ny = D.ny; H.nz = D.nz; H.N = D.N; H.F = D.F; H.syz = D.syz;
    H.vc.resize(D.N);
    MB_CUDA(cudaMemcpy(H.vc.data(), c->vcode, 4 * D.N, cudaMemcpyDeviceToHost));
    if (D.F) {
        H.pg.resize(D.F); H.pe.resize(D.F);
        MB_CUDA(cudaMemcpy(H.pg.data(), c->pf_g, 4 * D.F, cudaMemcpyDeviceToHost));
        MB_CUDA(cudaMemcpy(H.pe.data(), c->pf_e, 4 * D.F, cudaMemcpyDeviceToHost));
    }
    const int64_t N = D.N, n = c->n;
    const int Nr = dd->n_r, Mbv = dd->n_bv, M1c = dd->n_1c, M = Mbv + M1c;
    const double A = c->P.A, invF = c->P.invF, tp = c->prm.E_tplus;
    // plating faces touching each voxel (as graphite or electrolyte voxel)
    std::vector<std::vector<int64_t>> vfaces(N);
    for (int64_t f = 0; f < D.F; ++f) {
        vfaces[H.pg[f]].push_back(f);
        vfaces[H.pe[f]].push_back(f);
    }
    std::vector<std::vector<Term>> prog(M);
    std::vector<int64_t> closure;
    auto add_vox = [&](int64_t v) {
        closure.push_back(v);
        closure.push_back(N + v);
    };
    for (int m = 0; m < M; ++m) {
        const bool bv = m < Mbv;
        const int64_t p = bv ? dd->p_bv[m] : dd->p_1c[m - Mbv];
        if (p < 0 || p >= n) return MB_EINVAL;
        std::vector<Term>& T = prog[m];
        if (p >= 2 * N) {                                 // face row of plating face f
            const int64_t f = p - 2 * N;
            closure.push_back(H.pg[f]); closure.push_back(N + H.pg[f]);
            closure.push_back(H.pe[f]); closure.push_back(N + H.pe[f]);
            closure.push_back(2 * N + f);
            if (bv) {
                Term t;
                t.type = T_GE;
                t.dof[0] = H.pg[f]; t.dof[1] = N + H.pg[f]; t.dof[2] = H.pe[f]; t.dof[3] = N + H.pe[f];
                t.dof[4] = 2 * N + f;
                t.wpl = invF;
                t.face = f;
                T.push_back(t);
            }
            continue;
        }
        const bool crow = p < N;
        const int64_t v = crow ? p : p - N;
        add_vox(v);
        for (int d = 0; d < 6; ++d) {
            int64_t w = H.nb(v, d);
            if (w >= 0) add_vox(w);
        }
        for (int64_t f : vfaces[v]) closure.push_back(2 * N + f);
        const int lv = H.phase(v);
        for (int d = 0; d < 6; ++d) {
            const int64_t w = H.nb(v, d);
            if (w < 0) continue;
            const int lw = H.phase(w);
            if (!bv) {
                if (lv == PE && lw == PE) {
                    Term t;
                    t.type = T_EE;
                    t.dof[0] = v; t.dof[2] = w;
                    t.wbv = crow ? tp * invF : 1.0;
                    T.push_back(t);
                }
                continue;
            }
            int64_t s, e;
            int dsol;
            bool solid_row;
            if (kinetic(lv) && lw == PE) { s = v; e = w; dsol = d; solid_row = true; }
            else if (lv == PE && kinetic(lw)) { s = w; e = v; dsol = d ^ 1; solid_row = false; }
            else continue;
            const int ls = H.phase(s);
            Term t;
            t.type = ls == PG ? T_GE : (ls == PK ? T_KE : T_LE);
            if (ls != PL) { t.dof[0] = s; t.dof[2] = e; }
            t.dof[1] = N + s; t.dof[3] = N + e;
            if (ls == PG) {
                t.face = H.iface(s, dsol);
                t.dof[4] = 2 * N + t.face;
            }
            if (crow) {
                if (solid_row) t.wbv = ls == PL ? 0.0 : A * invF;
                else { t.wbv = -A * invF; t.wpl = ls == PG ? -A * invF : 0.0; }
            } else {
                t.wbv = solid_row ? A : -A;
                t.wpl = ls == PG ? t.wbv : 0.0;
            }
            T.push_back(t);
        }
        if ((int)T.size() > TMAX) return MB_EINVAL;
    }
    std::sort(closure.begin(), closure.end());
    closure.erase(std::unique(closure.begin(), closure.end()), closure.end());
    const int nloc = (int)closure.size();
    std::map<int64_t, int> slot;
    for (int k = 0; k < nloc; ++k) slot[closure[k]] = k;
    // gated faces
    std::map<int64_t, int> gslot;
    std::vector<int32_t> gface;
    // term arrays
    std::vector<int8_t> ttype((size_t)M * TMAX, T_NONE), tgpos((size_t)M * TMAX * 5, 0);
    std::vector<int32_t> tidx((size_t)M * TMAX * 5, -1), tgate((size_t)M * TMAX, -1), gidx((size_t)M * GMAX, -1);
    std::vector<double> twbv((size_t)M * TMAX, 0.0), twpl((size_t)M * TMAX, 0.0);
    for (int m = 0; m < M; ++m) {
        std::vector<int32_t> glist;
        for (size_t t = 0; t < prog[m].size(); ++t) {
            const Term& T = prog[m][t];
            const size_t q = (size_t)m * TMAX + t;
            ttype[q] = (int8_t)T.type;
            twbv[q] = T.wbv;
            twpl[q] = T.wpl;
            for (int k = 0; k < 5; ++k) {
                if (T.dof[k] < 0) continue;
                const int s = slot.at(T.dof[k]);
                tidx[q * 5 + k] = s;
                auto it = std::find(glist.begin(), glist.end(), s);
                int pos = (int)(it - glist.begin());
                if (it == glist.end()) glist.push_back(s);
                if (pos >= GMAX) return MB_EINVAL;
                tgpos[q * 5 + k] = (int8_t)pos;
            }
            if (T.face >= 0) {
                auto it = gslot.find(T.face);
                int gs;
                if (it == gslot.end()) {
                    gs = (int)gface.size() / 3;
                    gslot[T.face] = gs;
                    gface.push_back(slot.at(N + H.pg[T.face]));
                    gface.push_back(slot.at(N + H.pe[T.face]));
                    gface.push_back(slot.at(2 * N + T.face));
                } else {
                    gs = it->second;
                }
                tgate[q] = gs;
            }
        }
        if ((int)glist.size() > GMAX) return MB_EINVAL;
        for (size_t e = 0; e < glist.size(); ++e) gidx[(size_t)m * GMAX + e] = glist[e];
    }
    // basis at the closure
    std::vector<double> UlocC((size_t)Nr * nloc), UlocR((size_t)nloc * Nr), us(nloc);
    for (int k = 0; k < nloc; ++k) {
        const int64_t dof = closure[k];
        for (int j = 0; j < Nr; ++j) {
            const double u = dd->U[(size_t)dof * Nr + j];
            UlocC[(size_t)j * nloc + k] = u;
            UlocR[(size_t)k * Nr + j] = u;
        }
        if (dof < N) us[k] = c->P.cref[H.phase(dof)];
        else if (dof < 2 * N) us[k] = 1.0;
        else us[k] = c->P.nc;
    }
    std::vector<double> P((size_t)Nr * M);
    for (int i = 0; i < Nr; ++i) {
        for (int m = 0; m < Mbv; ++m) P[(size_t)i * M + m] = dd->Pbv[(size_t)i * Mbv + m];
        for (int m = 0; m < M1c; ++m) P[(size_t)i * M + Mbv + m] = dd->P1c[(size_t)i * M1c + m];
    }
    // upload
    RomDev& d = R->d;
    d.Nr = Nr; d.Mbv = Mbv; d.M1c = M1c; d.M = M; d.nloc = nloc; d.ngate = (int)gface.size() / 3;
    auto up = [&](auto*& dst, const auto& src) -> bool {
        using T = typename std::remove_reference<decltype(src[0])>::type;
        using U = typename std::remove_const<T>::type;
        dst = rom_alloc<U>(R->owned, src.size());
        if (!dst) return false;
        return cudaMemcpy(dst, src.data(), sizeof(U) * src.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    };
    auto upr = [&](double*& dst, const double* src, size_t cnt) -> bool {
        dst = rom_alloc<double>(R->owned, cnt);
        if (!dst) return false;
        return cudaMemcpy(dst, src, 8 * cnt, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    bool ok = up(d.UlocR, UlocR) && up(d.us, us) && up(d.ttype, ttype) &&
              up(d.tidx, tidx) && up(d.twbv, twbv) && up(d.twpl, twpl) && up(d.tgate, tgate) &&
              up(d.tgpos, tgpos) && up(d.gidx, gidx) && up(d.P, P) &&
              upr(d.Ms, dd->Ms, (size_t)Nr * Nr) && upr(d.Alin, dd->Alin, (size_t)Nr * Nr) &&
              upr(d.bbnd, dd->bbnd, Nr) && upr(d.scp, dd->s_cp, Nr) && upr(d.sac, dd->s_ac, Nr) &&
              upr(d.a0, dd->a0, Nr);
    if (ok && !gface.empty()) ok = up(d.gface, gface);
    auto updf = [&](float2*& dst, const double* src, size_t cnt) -> bool {
        std::vector<float2> h(cnt ? cnt : 1);
        for (size_t i = 0; i < cnt; ++i) h[i] = df_from_double(src[i]);
        dst = rom_alloc<float2>(R->owned, h.size());
        if (!dst) return false;
        return cudaMemcpy(dst, h.data(), 8 * h.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (ok)
        ok = updf(d.Pdf, P.data(), P.size()) && updf(d.Msdf, dd->Ms, (size_t)Nr * Nr) &&
             updf(d.Alindf, dd->Alin, (size_t)Nr * Nr);
    // FP32 copies for the Newton matrix and the step-length norm
    auto upf = [&](float*& dst, const double* src, size_t cnt) -> bool {
        std::vector<float> h(src, src + cnt);
        dst = rom_alloc<float>(R->owned, cnt);
        if (!dst) return false;
        return cudaMemcpy(dst, h.data(), 4 * (cnt ? cnt : 1), cudaMemcpyHostToDevice) == cudaSuccess;
    };
    if (ok) {
        std::vector<float2> h(UlocC.size());
        for (size_t i = 0; i < h.size(); ++i) h[i] = df_from_double(UlocC[i]);
        d.UlocCdf = rom_alloc<float2>(R->owned, h.size());
        ok = d.UlocCdf && cudaMemcpy(d.UlocCdf, h.data(), 8 * (h.size() ? h.size() : 1), cudaMemcpyHostToDevice) ==
                               cudaSuccess;
    }
    if (ok) {
        std::vector<double> Pt((size_t)M * Nr);
        for (int i = 0; i < Nr; ++i)
            for (int k = 0; k < M; ++k) Pt[(size_t)k * Nr + i] = P[(size_t)i * M + k];
        ok = upf(d.Ptf, Pt.data(), Pt.size());
    }
    // the tcgen05 GEMM's operand (models with N_r <= 256; others keep the mma.sync kernel)
    if (ok && !t5_prepare(d, R->owned)) {
        d.Pbf = d.Psf = nullptr;
        cudaGetLastError();
    }
    if (ok)
        ok = upf(d.Msf, dd->Ms, (size_t)Nr * Nr) &&
             upf(d.Alinf, dd->Alin, (size_t)Nr * Nr) && upf(d.UlocRf, UlocR.data(), UlocR.size()) &&
             upf(d.UlocCf, UlocC.data(), UlocC.size()) && upf(d.usf, us.data(), us.size());
    if (ok) {
        // the step-length cap: voxel slots in their scales, face slots (-1)
        // relative to max(n_c, |n|) of the current reconstruction
        std::vector<double> usc(us);
        for (int64_t k = 0; k < nloc; ++k)
            if (closure[k] >= 2 * N) usc[k] = -1.0;
        ok = upf(d.uscf, usc.data(), usc.size());
        d.ncf = (float)c->P.nc;
    }
    // shared memory of the LU kernels beyond the default 48 KB
    if (ok)
        ok = cudaFuncSetAttribute(k_rom_lu<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ROM_LU_SMEM) == cudaSuccess &&
             cudaFuncSetAttribute(k_rom_lu<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ROM_LU_SMEM) == cudaSuccess &&
             cudaFuncSetAttribute(k_rom_lu<float, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ROM_LU_SMEM) == cudaSuccess &&
             cudaFuncSetAttribute(k_rom_lu<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ROM_LU_SMEM) == cudaSuccess &&
             cudaFuncSetAttribute(k_rom_lu<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ROM_LU_SMEM) == cudaSuccess &&
             cudaFuncSetAttribute(k_rom_lu<float, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  ROM_LU_SMEM) == cudaSuccess &&
             cudaFuncSetAttribute(k_rom_gmres, cudaFuncAttributeMaxDynamicSharedMemorySize, ROM_LU_SMEM) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(k_rom_gu, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(float) * GMAX * ROM_NR_MAX)) == cudaSuccess;
    if (!ok) return cuda_fail(cudaGetLastError(), "rom upload");
    return MB_OK;
}

static int rom_work_alloc(mb_rom* R, int B) {
    RomWork& w = R->w;
    const RomDev& d = R->d;
    rom_work_free(w);
    w.B = B;
    auto& L = w.bufs;
    w.a = rom_alloc<double>(L, (size_t)B * d.Nr);
    w.a_old = rom_alloc<double>(L, (size_t)B * d.Nr);
    w.delta = rom_alloc<double>(L, (size_t)B * d.Nr);
    w.r = rom_alloc<double>(L, (size_t)B * d.Nr);
    w.J = rom_alloc<float>(L, (size_t)B * d.Nr * d.Nr);
    w.uloc = rom_alloc<double>(L, (size_t)B * d.nloc);
    w.uloc_old = rom_alloc<double>(L, (size_t)B * d.nloc);
    w.f = rom_alloc<double>(L, (size_t)B * d.M);
    w.G = rom_alloc<float>(L, (size_t)B * (d.M ? d.M : 1) * GMAX);
    w.dpart = rom_alloc<float>(L, (size_t)2 * B * ((d.nloc + UN_K - 1) / UN_K));
    w.hp = rom_alloc<int>(L, B);
    w.hplist = rom_alloc<int>(L, B);
    w.alist = rom_alloc<int>(L, B);
    w.pit = rom_alloc<int>(L, B);
    w.dnprev = rom_alloc<float>(L, B);
    w.G64 = rom_alloc<double>(L, (size_t)B * (d.M ? d.M : 1) * GMAX);
    w.GU64 = rom_alloc<double>(L, (size_t)B * (d.M ? d.M : 1) * d.Nr);
    w.J64 = rom_alloc<double>(L, (size_t)B * d.Nr * d.Nr);
    w.lpiv = rom_alloc<int>(L, (size_t)B * d.Nr);
    w.lsc = rom_alloc<float>(L, (size_t)B * 2 * d.Nr);
    w.GU = rom_alloc<float>(L, (size_t)B * (d.M ? d.M : 1) * d.Nr);
    w.prm = rom_alloc<double>(L, (size_t)B * RP);
    w.gate = rom_alloc<uint8_t>(L, (size_t)B * (d.ngate ? d.ngate : 1));
    w.gate2 = rom_alloc<uint8_t>(L, (size_t)B * (d.ngate ? d.ngate : 1));
    w.active = rom_alloc<int>(L, B);
    w.failed = rom_alloc<int>(L, B);
    w.pass_on = rom_alloc<int>(L, B);
    w.counts = rom_alloc<int>(L, 4);
    w.ctl = rom_alloc<int>(L, 4);
    w.tcerr = rom_alloc<int>(L, 4);
    w.its = rom_alloc<long long>(L, B);
    w.flips = rom_alloc<long long>(L, B);
    w.V = rom_alloc<double>(L, (size_t)B);
    w.S = rom_alloc<double>(L, (size_t)B);
    w.a_hold = rom_alloc<double>(L, (size_t)B * d.Nr);
    w.retry = rom_alloc<int>(L, B);
    for (void* p : L)
        if (!p) { rom_work_free(w); return MB_ENOMEM; }
    return MB_OK;
}

// ------------------------------------------------------------ slot batch
// A batch of B slots; an empty slot is marked failed and skipped by every
// kernel.  Each occupied slot advances one time step per rom_batch_step.
int rom_batch_alloc(mb_rom* R, int B) {
    RomWork& w = R->w;
    // a batch of the same size reuses the buffers (and with them the captured step graph)
    if (!(w.B == B && !w.bufs.empty())) {
        int rc = rom_work_alloc(R, B);
        if (rc) return rc;
    }
    cudaStream_t s = R->cell->stream;
    std::vector<int> ones(B, 1);
    MB_CUDA(cudaMemcpyAsync(w.failed, ones.data(), 4 * B, cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemsetAsync(w.a, 0, 8 * (size_t)B * R->d.Nr, s));
    MB_CUDA(cudaMemsetAsync(w.prm, 0, 8 * (size_t)B * RP, s));
    MB_CUDA(cudaMemsetAsync(w.gate, 0, (size_t)B * (R->d.ngate ? R->d.ngate : 1), s));
    MB_CUDA(cudaMemsetAsync(w.its, 0, 8 * B, s));
    MB_CUDA(cudaMemsetAsync(w.flips, 0, 8 * B, s));
    MB_CUDA(cudaMemsetAsync(w.hp, 0, 4 * B, s));
    MB_CUDA(cudaMemsetAsync(w.pit, 0, 4 * B, s));
    MB_CUDA(cudaMemsetAsync(w.tcerr, 0, 16, s));
    MB_CUDA(cudaStreamSynchronize(s));
    w.hp_any = 0;
    return MB_OK;
}

int rom_slot_start(mb_rom* R, int b, const mb_rom_params& p, double dt) {
    RomWork& w = R->w;
    k_rom_slot_start<<<1, 128, 0, R->cell->stream>>>(R->d, b, p.I_app, p.s_i0, p.k_pl, 1.0 / dt, w.a, w.prm,
                                                     w.failed, w.its, w.flips, w.hp), count_launch(R->cell);
    MB_CUDA_LAUNCH("rom_slot_start");
    return MB_OK;
}

int rom_slot_clear(mb_rom* R, int b) {
    int one = 1;
    MB_CUDA(cudaMemcpyAsync(R->w.failed + b, &one, 4, cudaMemcpyHostToDevice, R->cell->stream));
    MB_CUDA(cudaStreamSynchronize(R->cell->stream));
    return MB_OK;
}

// current outputs of every slot (host arrays of B)
int rom_batch_outputs(mb_rom* R, double* hV, double* hS, int* hfailed) {
    RomWork& w = R->w;
    cudaStream_t s = R->cell->stream;
    const int B = w.B;
    k_rom_outputs<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(R->d, B, w.a, w.V, w.S), count_launch(R->cell);
    MB_CUDA(cudaMemcpyAsync(hV, w.V, 8 * B, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaMemcpyAsync(hS, w.S, 8 * B, cudaMemcpyDeviceToHost, s));
    if (hfailed) MB_CUDA(cudaMemcpyAsync(hfailed, w.failed, 4 * B, cudaMemcpyDeviceToHost, s));
    int terr = 0;
    MB_CUDA(cudaMemcpyAsync(&terr, w.tcerr, 4, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    if (terr) {
        R->d.tc = 1;   // the tcgen05 GEMM gave up waiting: the mma.sync kernel from now on
        set_error("reduced model: a bounded wait of the tcgen05 Newton-matrix GEMM gave up");
        return MB_ETIMEOUT;
    }
    return MB_OK;
}

int rom_slot_stats(mb_rom* R, int b, long long* its, long long* flips, double* a) {
    cudaStream_t s = R->cell->stream;
    if (its) MB_CUDA(cudaMemcpyAsync(its, R->w.its + b, 8, cudaMemcpyDeviceToHost, s));
    if (flips) MB_CUDA(cudaMemcpyAsync(flips, R->w.flips + b, 8, cudaMemcpyDeviceToHost, s));
    if (a) MB_CUDA(cudaMemcpyAsync(a, R->w.a + (size_t)b * R->d.Nr, 8 * R->d.Nr, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    return MB_OK;
}

// ---- the kernels of one reduced time step, by phase.  Host mode launches
// the escalated-instance kernels over the counted lists; graph mode launches
// them for the whole batch (the lists end at -1) and reads the Newton
// iteration and pass numbers from device memory.
// the step's start: a_old = a, its reconstruction and gates, every slot's pass on
static void step_begin(mb_rom* R, cudaStream_t s) {
    mb_cell* c = R->cell;
    const RomDev& d = R->d;
    RomWork& w = R->w;
    const int B = w.B;
    const unsigned nb = (unsigned)(((int64_t)B * d.Nr + 255) / 256);
    const unsigned bb = (unsigned)((B + 255) / 256);
    const dim3 gg((unsigned)((d.nloc + 255) / 256), (unsigned)B);
    const unsigned gt = (unsigned)(((int64_t)(d.ngate ? d.ngate : 1) * B + 255) / 256);
    k_rom_copy<<<nb, 256, 0, s>>>(d.Nr, B, nullptr, w.a, w.a_old), count_launch(c);
    k_rom_gather<<<gg, 256, 0, s>>>(d, w.a_old, w.uloc_old, nullptr), count_launch(c);
    if (d.ngate)
        k_rom_gate<<<gt, 256, 0, s>>>(d, B, w.uloc_old, w.uloc_old, GATE_N_REL * c->P.nc, w.gate), count_launch(c);
    k_rom_set_active<<<bb, 256, 0, s>>>(B, nullptr, w.failed, w.pass_on, nullptr, w.hp), count_launch(c);
}

// a pass's start: its slots restart from a_old
static void pass_begin(mb_rom* R, cudaStream_t s) {
    mb_cell* c = R->cell;
    const RomDev& d = R->d;
    RomWork& w = R->w;
    const int B = w.B;
    const unsigned nb = (unsigned)(((int64_t)B * d.Nr + 255) / 256);
    const unsigned bb = (unsigned)((B + 255) / 256);
    k_rom_copy<<<nb, 256, 0, s>>>(d.Nr, B, w.pass_on, w.a_old, w.a), count_launch(c);
    k_rom_set_active<<<bb, 256, 0, s>>>(B, w.pass_on, w.failed, w.active, w.pit, nullptr), count_launch(c);
}

static bool rom_refine(const RomDev& d) {
    return d.ir && d.M > 0 && gmres_smem(d.Nr, d.M, GMRES_M) <= (size_t)ROM_LU_SMEM;
}

// escalated instances, part A: FP64 interpolated terms and derivatives, G U_loc in
// FP64 (and, without refinement, their FP64 Newton matrices)
static void iter_hp_a(mb_rom* R, cudaStream_t s, int nhp, bool graph) {
    mb_cell* c = R->cell;
    const RomDev& d = R->d;
    RomWork& w = R->w;
    const int n = graph ? w.B : nhp;
    k_rom_ei<true><<<(unsigned)(((int64_t)d.M * n + 127) / 128), 128, 0, s>>>(
        d, c->P, c->Pf, n, w.uloc, w.gate, w.prm, w.active, w.hp, w.hplist, w.f, w.G, w.G64), count_launch(c);
    const unsigned gy = (unsigned)(graph ? std::min(n, 64) : n);
    if (rom_refine(d))
        k_rom_gu64<true><<<dim3((unsigned)d.M, gy), 64, 0, s>>>(d, w.G64, w.active, w.hp, w.hplist, n, w.GU64);
    else
        k_rom_gu64<false><<<dim3((unsigned)d.M, gy), 64, 0, s>>>(d, w.G64, w.active, w.hp, w.hplist, n, w.GU64);
    count_launch(c);
    if (!rom_refine(d))
        k_rom_jac64<<<dim3((unsigned)d.Nr, gy), 128, 0, s>>>(d, w.prm, w.GU64, w.active, w.hp, w.hplist, n, w.J64),
            count_launch(c);
}

// escalated instances, part B: their Newton steps (GMRES on FP64 products, or the FP64 LU)
static void iter_hp_b(mb_rom* R, cudaStream_t s, int nhp, bool graph) {
    mb_cell* c = R->cell;
    const RomDev& d = R->d;
    RomWork& w = R->w;
    const int n = graph ? w.B : nhp;
    if (rom_refine(d))
        k_rom_gmres<<<(unsigned)n, 256, gmres_smem(d.Nr, d.M, GMRES_M), s>>>(
            d, w.prm, w.GU64, w.r, w.J, w.lpiv, w.lsc, w.active, w.hp, w.hplist, GMRES_M, GMRES_CYCLES, GMRES_ETA,
            w.delta), count_launch(c);
    else
        launch_rom_lu<double>(d.Nr, n, w.J64, w.r, w.active, w.hp, 1, w.hplist, w.delta, s), count_launch(c);
}

// one reduced Newton iteration of the active slots.  Host mode: hp_any and the
// list length n_alist come from the host's last count; graph mode: the
// escalated parts are left to the caller (conditional nodes) and the GEMM
// reads the iteration number and the list length from device memory.
static void iter_main_a(mb_rom* R, cudaStream_t s) {
    mb_cell* c = R->cell;
    const RomDev& d = R->d;
    RomWork& w = R->w;
    const int B = w.B;
    const dim3 gg((unsigned)((d.nloc + 255) / 256), (unsigned)B);
    k_rom_gather<<<gg, 256, 0, s>>>(d, w.a, w.uloc, w.active), count_launch(c);
    if (d.M)
        k_rom_ei<false><<<(unsigned)(((int64_t)d.M * B + 127) / 128), 128, 0, s>>>(
            d, c->P, c->Pf, B, w.uloc, w.gate, w.prm, w.active, w.hp, w.hplist, w.f, w.G, w.G64), count_launch(c);
}
// the Newton-matrix GEMM in variant tc (0 FP32 FMA, 1 mma.sync 3xTF32, 2 tcgen05 3xTF32)
static void launch_rom_jac_p(const RomDev& d, cudaStream_t s, int tc, int B, int ncols, const int* al,
                             const double* prm, const float* GU, const int* hp, float* J, const int* dit,
                             const int* dn, int* tcerr) {
    const dim3 gj((unsigned)(((int64_t)ncols * d.Nr + JT_COLS - 1) / JT_COLS), (unsigned)((d.Nr + JT_ROWS - 1) / JT_ROWS));
    if (tc == 2 && d.Pbf)
        k_rom_jac5<<<(unsigned)(((int64_t)ncols * d.Nr + T5_M - 1) / T5_M), T5_THREADS, T5_SMEM, s>>>(
            d, B, ncols, al, prm, GU, hp, J, dit, dn, tcerr);
    else if (tc)
        k_rom_jac<true><<<gj, 256, 0, s>>>(d, B, ncols, al, prm, GU, hp, J, dit, dn);
    else
        k_rom_jac<false><<<gj, 256, 0, s>>>(d, B, ncols, al, prm, GU, hp, J, dit, dn);
}
static void launch_rom_jac(mb_rom* R, cudaStream_t s, int tc, int ncols, const int* al, const int* dit,
                           const int* dn) {
    RomWork& w = R->w;
    launch_rom_jac_p(R->d, s, tc, w.B, ncols, al, w.prm, w.GU, w.hp, w.J, dit, dn, w.tcerr);
}

// Autotuning of the Newton-matrix GEMM: once per model shape (N_r, M), every
// variant the model admits is timed on a scratch batch of TUNE_B instances
// (GU zeroed; one warm-up and three timed launches, CUDA events on the
// cell's stream) and the fastest is kept for every later batch of that
// shape, whatever its size: the variant, and so the rounding of the Newton
// matrices, depends on the model only, so an instance gives the same result
// alone or in any batch.  The three variants give FP32-accurate matrices
// (tested against each other to 1e-9 on reduced trajectories).
constexpr int TUNE_B = 256;
struct TuneRec {
    int choice;
    float ms[3];
};
static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, TuneRec> g_tune;

static int rom_tune_gemm(mb_rom* R) {
    const RomDev& d = R->d;
    if (R->tc_forced || d.M == 0) return MB_OK;
    const auto key = std::make_pair(d.Nr, d.M);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            R->d.tc = it->second.choice;
            for (int k = 0; k < 3; ++k) R->tune_ms[k] = it->second.ms[k];
            return MB_OK;
        }
    }
    cudaStream_t s = R->cell->stream;
    const int Bt = TUNE_B;
    float *GU = nullptr, *J = nullptr;
    double* prm = nullptr;
    int *hp = nullptr, *terr_d = nullptr;
    cudaError_t e = cudaMalloc(&GU, sizeof(float) * (size_t)Bt * d.M * d.Nr);
    if (e == cudaSuccess) e = cudaMalloc(&J, sizeof(float) * (size_t)Bt * d.Nr * d.Nr);
    if (e == cudaSuccess) e = cudaMalloc(&prm, sizeof(double) * (size_t)Bt * RP);
    if (e == cudaSuccess) e = cudaMalloc(&hp, sizeof(int) * (size_t)Bt);
    if (e == cudaSuccess) e = cudaMalloc(&terr_d, 16);
    if (e == cudaErrorMemoryAllocation) {   // no room for the scratch batch: keep the default variant untuned
        cudaGetLastError();
        cudaFree(GU); cudaFree(J); cudaFree(prm); cudaFree(hp); cudaFree(terr_d);
        return MB_OK;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(GU, 0, sizeof(float) * (size_t)Bt * d.M * d.Nr, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(prm, 0, sizeof(double) * (size_t)Bt * RP, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hp, 0, sizeof(int) * (size_t)Bt, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(terr_d, 0, 16, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int best = d.tc;
    float best_ms = 1e30f;
    for (int tc = 0; tc <= 2 && e == cudaSuccess; ++tc) {
        R->tune_ms[tc] = -1.f;
        if (tc == 2 && !d.Pbf) continue;
        launch_rom_jac_p(d, s, tc, Bt, Bt, nullptr, prm, GU, hp, J, nullptr, nullptr, terr_d);
        cudaEventRecord(e0, s);
        for (int k = 0; k < 3; ++k) launch_rom_jac_p(d, s, tc, Bt, Bt, nullptr, prm, GU, hp, J, nullptr, nullptr, terr_d);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        int terr = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&terr, terr_d, 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        if (terr) {   // a bounded wait of the tcgen05 kernel gave up: not a candidate
            e = cudaMemset(terr_d, 0, 16);
            continue;
        }
        R->tune_ms[tc] = ms / 3.f;
        if (ms < best_ms) { best_ms = ms; best = tc; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(GU); cudaFree(J); cudaFree(prm); cudaFree(hp); cudaFree(terr_d);
    if (e != cudaSuccess) return cuda_fail(e, "reduced model: GEMM autotuning");
    MB_CUDA_LAUNCH("rom_tune_gemm");
    R->d.tc = best;
    TuneRec rec;
    rec.choice = best;
    for (int k = 0; k < 3; ++k) rec.ms[k] = R->tune_ms[k];
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = rec;
    return MB_OK;
}

static void iter_main_b(mb_rom* R, cudaStream_t s, bool listed, int ncols, const int* dit) {
    mb_cell* c = R->cell;
    const RomDev& d = R->d;
    RomWork& w = R->w;
    const int B = w.B;
    if (d.M)
        k_rom_gu<<<dim3((unsigned)d.M, (unsigned)((B + GU_INST - 1) / GU_INST)), 256, sizeof(float) * GMAX * d.Nr, s>>>(
            d, B, w.G, w.active, w.hp, w.GU),
            count_launch(c);
    if (ncols > 0) {
        const int* al = (listed || dit) ? w.alist : nullptr;
        const int* dn = dit ? w.counts + 2 : nullptr;
        launch_rom_jac(R, s, d.tc, ncols, al, dit, dn);
        count_launch(c);
    }
    k_rom_resid<<<(unsigned)B, 128, 0, s>>>(d, w.a, w.a_old, w.prm, w.f, w.active, w.r), count_launch(c);
    const bool refine = rom_refine(d);
    launch_rom_lu<float>(d.Nr, B, w.J, w.r, w.active, w.hp, 0, nullptr, w.delta, s, refine ? w.lpiv : nullptr,
                         refine ? w.lsc : nullptr),
        count_launch(c);
}
static void iter_main_c(mb_rom* R, cudaStream_t s) {
    mb_cell* c = R->cell;
    const RomDev& d = R->d;
    RomWork& w = R->w;
    const int B = w.B;
    const unsigned nkt = (unsigned)((d.nloc + UN_K - 1) / UN_K);
    k_rom_unorm<<<dim3(nkt, (unsigned)((B + UN_B - 1) / UN_B)), 256, 0, s>>>(d, B, w.delta, w.active, w.uloc,
                                                                             w.dpart),
        count_launch(c);
    k_rom_apply<<<(unsigned)B, 32, 0, s>>>(d, B, (int)nkt, w.a, w.delta, w.dpart, w.active, w.failed, w.its, w.pit,
                                           w.hp, w.dnprev, R->cell->opt.newton_rate_test), count_launch(c);
    k_rom_count_hp<<<1, 256, 0, s>>>(B, w.active, w.hp, w.counts, w.hplist, w.alist), count_launch(c);
}

// a pass's end: instances still iterating have failed; the gates are re-taken
// and the slots whose gates flipped take another pass (pass_on)
static void pass_end(mb_rom* R, cudaStream_t s, int last_pass, const int* dpass) {
    mb_cell* c = R->cell;
    const RomDev& d = R->d;
    RomWork& w = R->w;
    const int B = w.B;
    const unsigned bb = (unsigned)((B + 255) / 256);
    k_rom_fail_active<<<bb, 256, 0, s>>>(B, w.active, w.failed), count_launch(c);
    if (!d.ngate) return;
    const dim3 gg((unsigned)((d.nloc + 255) / 256), (unsigned)B);
    const unsigned gt = (unsigned)(((int64_t)d.ngate * B + 255) / 256);
    k_rom_gather<<<gg, 256, 0, s>>>(d, w.a, w.uloc, nullptr), count_launch(c);
    k_rom_gate<<<gt, 256, 0, s>>>(d, B, w.uloc, w.uloc_old, GATE_N_REL * c->P.nc, w.gate2), count_launch(c);
    k_rom_flips<<<(unsigned)B, 256, 0, s>>>(d.ngate, B, w.gate, w.gate2, w.failed, w.pass_on, w.flips, w.gate,
                                           last_pass, dpass), count_launch(c);
    k_rom_count<<<1, 256, 0, s>>>(B, w.pass_on, w.counts + 3), count_launch(c);
}

// one implicit Euler step of every occupied slot, driven from the host (a
// count read back after every Newton iteration and pass)
static int rom_batch_step_host(mb_rom* R) {
    mb_cell* c = R->cell;
    cudaStream_t s = c->stream;
    const RomDev& d = R->d;
    RomWork& w = R->w;
    const int B = w.B;
    step_begin(R, s);
    w.hp_any = 0;
    for (int pass = 1; pass <= ROM_PASSES; ++pass) {
        pass_begin(R, s);
        for (int it = 0; it < ROM_MAXIT; ++it) {
            // escalated-instance kernels only while some instance uses them (hp only turns on
            // within a step, so the count of the previous iteration covers this one)
            const int nhp = w.hp_any;
            iter_main_a(R, s);
            if (nhp > 0) iter_hp_a(R, s, nhp, false);
            // the first iteration of a pass: every instance; later: the listed active FP32 ones
            const bool listed = it > 0 && w.n_alist >= 0;
            iter_main_b(R, s, listed, listed ? w.n_alist : B, nullptr);
            if (nhp > 0) iter_hp_b(R, s, nhp, false);
            iter_main_c(R, s);
            int hc[3] = {0, 0, 0};
            MB_CUDA(cudaMemcpyAsync(hc, w.counts, 12, cudaMemcpyDeviceToHost, s));
            MB_CUDA(cudaStreamSynchronize(s));
            w.hp_any = hc[1];
            w.n_alist = hc[2];
            if (hc[0] == 0) break;
        }
        pass_end(R, s, pass == ROM_PASSES ? 1 : 0, nullptr);
        if (!d.ngate) break;
        int hcount = 0;
        MB_CUDA(cudaMemcpyAsync(&hcount, w.counts + 3, 4, cudaMemcpyDeviceToHost, s));
        MB_CUDA(cudaStreamSynchronize(s));
        if (hcount == 0) break;
    }
    MB_CUDA_LAUNCH("rom_step");
    return MB_OK;
}

// ---- graph mode: control kernels and the capture
__global__ void k_rom_ctl_step(int* ctl, int* counts) {
    ctl[1] = 0;       // passes done
    counts[1] = 0;    // no escalated instance at the start of a step
}
__global__ void k_rom_ctl_pass_begin(int* ctl, cudaGraphConditionalHandle h_it) {
    ctl[0] = 0;
    cudaGraphSetConditional(h_it, 1u);
}
__global__ void k_rom_ctl_iter_begin(const int* counts, cudaGraphConditionalHandle h_a, cudaGraphConditionalHandle h_b) {
    const unsigned v = counts[1] > 0 ? 1u : 0u;   // escalated instances at the last count
    cudaGraphSetConditional(h_a, v);
    cudaGraphSetConditional(h_b, v);
}
__global__ void k_rom_ctl_iter_end(int* ctl, const int* counts, cudaGraphConditionalHandle h_it) {
    const int it = ++ctl[0];
    cudaGraphSetConditional(h_it, (counts[0] > 0 && it < ROM_MAXIT) ? 1u : 0u);
}
__global__ void k_rom_ctl_pass_end(int* ctl, const int* counts, int ngate, cudaGraphConditionalHandle h_pass) {
    const int p = ++ctl[1];
    cudaGraphSetConditional(h_pass, (ngate && counts[3] > 0 && p < ROM_PASSES) ? 1u : 0u);
}

// a conditional handle of the graph being captured on s
static int cap_handle(cudaStream_t s, unsigned dflt, unsigned flags, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    MB_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr));
    if (st != cudaStreamCaptureStatusActive) { set_error("reduced step graph: capture not active"); return MB_ECUDA; }
    MB_CUDA(cudaGraphConditionalHandleCreate(h, g, dflt, flags));
    return MB_OK;
}
// a conditional node on handle h at the current point of the capture on s;
// *body is its body graph, to be filled by capturing another stream into it
static int cap_node(cudaStream_t s, cudaGraphConditionalNodeType type, cudaGraphConditionalHandle h,
                    cudaGraph_t* body) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    MB_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &ed, &nd));
    if (st != cudaStreamCaptureStatusActive) { set_error("reduced step graph: capture not active"); return MB_ECUDA; }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    MB_CUDA(cudaGraphAddNode(&node, g, deps, ed, nd, &np));
    *body = np.conditional.phGraph_out[0];
    MB_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return MB_OK;
}
static int cap_into(cudaStream_t s, cudaGraph_t body) {
    MB_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    return MB_OK;
}
static int cap_end(cudaStream_t s) {
    cudaGraph_t g = nullptr;
    MB_CUDA(cudaStreamEndCapture(s, &g));
    return MB_OK;
}

// The step as one graph (s0 the top level, s1..s3 fill the nested bodies):
//   step start; while (passes) { pass start; while (Newton iterations) {
//   gather and FP32-path terms; if (escalated) { part A }; GU, GEMM, residual,
//   FP32 LU; if (escalated) { part B }; step length, update, counts }; pass end }
// The loop and branch conditions are set by control kernels from the device
// counts, in the order in which the host-driven step takes its decisions.
static int rom_graph_capture(mb_rom* R, cudaStream_t s0, cudaStream_t s1, cudaStream_t s2, cudaStream_t s3) {
    RomWork& w = R->w;
    const RomDev& d = R->d;
    int rc;
    cudaGraphConditionalHandle h_pass, h_it, h_a, h_b;
    cudaGraph_t bp, bi, ba, bb;
    step_begin(R, s0);
    k_rom_ctl_step<<<1, 1, 0, s0>>>(w.ctl, w.counts);
    if ((rc = cap_handle(s0, 1u, cudaGraphCondAssignDefault, &h_pass))) return rc;
    if ((rc = cap_node(s0, cudaGraphCondTypeWhile, h_pass, &bp))) return rc;
    // pass body
    if ((rc = cap_into(s1, bp))) return rc;
    pass_begin(R, s1);
    if ((rc = cap_handle(s1, 0u, 0u, &h_it))) return rc;
    k_rom_ctl_pass_begin<<<1, 1, 0, s1>>>(w.ctl, h_it);
    if ((rc = cap_node(s1, cudaGraphCondTypeWhile, h_it, &bi))) return rc;
    // Newton iteration body
    if ((rc = cap_into(s2, bi))) return rc;
    if ((rc = cap_handle(s2, 0u, 0u, &h_a)) || (rc = cap_handle(s2, 0u, 0u, &h_b))) return rc;
    k_rom_ctl_iter_begin<<<1, 1, 0, s2>>>(w.counts, h_a, h_b);
    iter_main_a(R, s2);
    if ((rc = cap_node(s2, cudaGraphCondTypeIf, h_a, &ba))) return rc;
    if ((rc = cap_into(s3, ba))) return rc;
    iter_hp_a(R, s3, 0, true);
    if ((rc = cap_end(s3))) return rc;
    iter_main_b(R, s2, false, w.B, w.ctl);
    if ((rc = cap_node(s2, cudaGraphCondTypeIf, h_b, &bb))) return rc;
    if ((rc = cap_into(s3, bb))) return rc;
    iter_hp_b(R, s3, 0, true);
    if ((rc = cap_end(s3))) return rc;
    iter_main_c(R, s2);
    k_rom_ctl_iter_end<<<1, 1, 0, s2>>>(w.ctl, w.counts, h_it);
    if ((rc = cap_end(s2))) return rc;
    // rest of the pass body
    pass_end(R, s1, 0, w.ctl + 1);
    k_rom_ctl_pass_end<<<1, 1, 0, s1>>>(w.ctl, w.counts, d.ngate, h_pass);
    if ((rc = cap_end(s1))) return rc;
    (void)bi;
    return MB_OK;
}

static int rom_graph_build(mb_rom* R) {
    mb_cell* c = R->cell;
    cudaStream_t s0 = c->stream, aux[3] = {nullptr, nullptr, nullptr};
    for (auto& a : aux) MB_CUDA(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
    const int64_t saved = c->launches;
    int rc = MB_OK;
    if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "reduced step graph: begin capture");
    } else {
        rc = rom_graph_capture(R, s0, aux[0], aux[1], aux[2]);
        // end every capture still open (after a failure), innermost first
        for (int k = 2; k >= 0; --k) {
            cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
            cudaStreamIsCapturing(aux[k], &st);
            if (st != cudaStreamCaptureStatusNone) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(aux[k], &g);
            }
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s0, &g);
        if (!rc && (e != cudaSuccess || !g)) rc = cuda_fail(e, "reduced step graph: end capture");
        if (!rc && cudaGraphInstantiate(&R->w.gexec, g, 0) != cudaSuccess)
            rc = cuda_fail(cudaGetLastError(), "reduced step graph: instantiate");
        if (g) cudaGraphDestroy(g);
    }
    c->launches = saved;
    for (auto& a : aux) cudaStreamDestroy(a);
    if (rc) {
        R->w.gexec = nullptr;
        cudaGetLastError();
    }
    return rc;
}

// one implicit Euler step of every occupied slot (reduced Newton with the
// plating active-set passes); a slot whose Newton iteration fails is marked
// failed (and skipped from then on).  By default the whole step is one CUDA
// graph launch (built at the batch's first step); without it (or if it cannot
// be built) the host drives the loops.
int rom_batch_step(mb_rom* R) {
    RomWork& w = R->w;
    if (R->d.graph && !w.graph_failed) {
        if (w.gexec && (w.g_tc != R->d.tc || w.g_ir != R->d.ir || w.g_rate != R->cell->opt.newton_rate_test)) {
            cudaGraphExecDestroy(w.gexec);   // captured with other kernels or arguments
            w.gexec = nullptr;
        }
        if (!w.gexec) {
            if (rom_graph_build(R)) w.graph_failed = true;
            w.g_tc = R->d.tc;
            w.g_ir = R->d.ir;
            w.g_rate = R->cell->opt.newton_rate_test;
        }
        if (w.gexec) {
            MB_CUDA(cudaGraphLaunch(w.gexec, R->cell->stream));
            count_launch(R->cell);
            return MB_OK;
        }
    }
    return rom_batch_step_host(R);
}

}  // namespace mb

using namespace mb;

extern "C" int mb_rom_create(mb_cell* cell, const mb_rom_data* d, mb_rom** out) {
    if (!cell || !d || !out || d->n_r < 1 || d->n_r > ROM_NR_MAX || d->n_bv < 0 || d->n_1c < 0 || !d->U ||
        !d->Ms || !d->Alin || !d->bbnd || !d->s_cp || !d->s_ac || !d->a0 || (d->n_bv && (!d->p_bv || !d->Pbv)) ||
        (d->n_1c && (!d->p_1c || !d->P1c))) {
        set_error("mb_rom_create: invalid argument");
        return MB_EINVAL;
    }
    mb_rom* R = new mb_rom();
    R->cell = cell;
    R->hU.assign(d->U, d->U + (size_t)cell->n * d->n_r);
    int rc = rom_build_host(R, d);
    if (rc) {
        if (rc == MB_EINVAL) set_error("mb_rom_create: point outside the residual or too many terms per point");
        for (void* p : R->owned) cudaFree(p);
        delete R;
        return rc;
    }
    *out = R;
    return MB_OK;
}

extern "C" int mb_rom_dims(mb_rom* R, int* n_r, int* n_bv, int* n_1c) {
    if (!R) { set_error("mb_rom_dims: invalid argument"); return MB_EINVAL; }
    if (n_r) *n_r = R->d.Nr;
    if (n_bv) *n_bv = R->d.Mbv;
    if (n_1c) *n_1c = R->d.M1c;
    return MB_OK;
}

extern "C" int mb_rom_block_dims(mb_rom* R, int* n_c, int* n_n, int* n_phi) {
    if (!R) { set_error("mb_rom_block_dims: invalid argument"); return MB_EINVAL; }
    const int64_t N = R->cell->D.N, n = R->cell->n;
    const int Nr = R->d.Nr;
    int cnt[3] = {0, 0, 0};
    for (int k = 0; k < Nr; ++k) {
        int f = -1;
        for (int64_t i = 0; i < n; ++i)
            if (R->hU[(size_t)i * Nr + k] != 0.0) {
                const int fi = est_field(i, N);
                f = (f < 0 || f == fi) ? fi : 3;
            }
        if (f >= 0 && f < 3) ++cnt[f];
    }
    if (n_c) *n_c = cnt[0];
    if (n_phi) *n_phi = cnt[1];
    if (n_n) *n_n = cnt[2];
    return MB_OK;
}

extern "C" int mb_rom_destroy(mb_rom* R) {
    if (!R) { set_error("mb_rom_destroy: invalid argument"); return MB_EINVAL; }
    rom_work_free(R->w);
    for (void* p : R->est.bufs) cudaFree(p);
    for (void* p : R->owned) cudaFree(p);
    delete R;
    return MB_OK;
}

namespace mb {
// B slots started at the initial coefficients with the instance parameters prm
static int rom_batch_begin(mb_rom* R, int B, const mb_rom_params* prm, double dt) {
    int rc = rom_batch_alloc(R, B);
    if (rc) { set_error("reduced model: device memory for the batch"); return rc; }
    // every instance's parameters in one copy, then one start kernel
    std::vector<double> hp((size_t)RP * B);
    for (int b = 0; b < B; ++b) {
        hp[(size_t)RP * b] = prm[b].I_app;
        hp[(size_t)RP * b + 1] = prm[b].s_i0;
        hp[(size_t)RP * b + 2] = prm[b].k_pl;
        hp[(size_t)RP * b + 3] = 1.0 / dt;
    }
    RomWork& w = R->w;
    cudaStream_t s = R->cell->stream;
    MB_CUDA(cudaMemcpyAsync(w.prm, hp.data(), 8 * hp.size(), cudaMemcpyHostToDevice, s));
    w.hprm = hp;
    const int64_t n = (int64_t)B * R->d.Nr;
    k_rom_batch_start<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
        R->d, B, w.a, w.failed, w.its, w.flips, w.hp), count_launch(R->cell);
    MB_CUDA_LAUNCH("rom_batch_start");
    MB_CUDA(cudaStreamSynchronize(s));   // the host parameter buffer goes out of scope
    return rom_tune_gemm(R);
}
}  // namespace mb

static int rom_solve(mb_rom* R, int B, const mb_rom_params* prm, int n_steps, double dt, double* V_out,
                     double* sac_out, double* a_final, double* a_traj, mb_rom_info* info);

extern "C" int mb_rom_solve_batch(mb_rom* R, int B, const mb_rom_params* prm, int n_steps, double dt, double* V_out,
                                  double* sac_out, double* a_final, mb_rom_info* info) {
    if (!R || B < 1 || !prm || n_steps < 0 || !(dt > 0) || !V_out || !sac_out) {
        set_error("mb_rom_solve_batch: invalid argument");
        return MB_EINVAL;
    }
    return rom_solve(R, B, prm, n_steps, dt, V_out, sac_out, a_final, nullptr, info);
}

extern "C" int mb_rom_solve_batch_traj(mb_rom* R, int B, const mb_rom_params* prm, int n_steps, double dt,
                                       double* V_out, double* sac_out, double* a_traj, mb_rom_info* info) {
    if (!R || B < 1 || !prm || n_steps < 0 || !(dt > 0) || !V_out || !sac_out || !a_traj) {
        set_error("mb_rom_solve_batch_traj: invalid argument");
        return MB_EINVAL;
    }
    return rom_solve(R, B, prm, n_steps, dt, V_out, sac_out, nullptr, a_traj, info);
}

extern "C" int mb_rom_basis(mb_rom* R, double* U) {
    if (!R || !U) { set_error("mb_rom_basis: invalid argument"); return MB_EINVAL; }
    memcpy(U, R->hU.data(), sizeof(double) * R->hU.size());
    return MB_OK;
}

namespace mb {
// One time step of every occupied slot with dt halving, as the full-order
// step does: the instances whose reduced Newton failed in the step restart
// from the state before it and take 2^h steps of dt / 2^h (h = 1 ..
// max_halvings, all in the same batch, the other slots held as failed
// meanwhile); an instance fails only when the smallest substeps fail too.
int rom_step_halving(mb_rom* R, int max_halvings) {
    RomWork& w = R->w;
    const int B = w.B, Nr = R->d.Nr;
    cudaStream_t s = R->cell->stream;
    const unsigned nb = (unsigned)(((int64_t)B * Nr + 255) / 256);
    std::vector<int> f0(B), f1(B);
    if (max_halvings > 0) {
        MB_CUDA(cudaMemcpyAsync(f0.data(), w.failed, 4 * B, cudaMemcpyDeviceToHost, s));
        MB_CUDA(cudaMemcpyAsync(w.a_hold, w.a, 8 * (size_t)B * Nr, cudaMemcpyDeviceToDevice, s));
    }
    int rc = rom_batch_step(R);
    if (rc || max_halvings <= 0) return rc;
    MB_CUDA(cudaMemcpyAsync(f1.data(), w.failed, 4 * B, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    std::vector<int> retry(B, 0);
    int nretry = 0;
    for (int b = 0; b < B; ++b)
        if (f1[b] && !f0[b]) { retry[b] = 1; ++nretry; }
    if (!nretry) return MB_OK;
    std::vector<double> hp = w.hprm;
    for (int h = 1; h <= max_halvings && nretry; ++h) {
        // retried slots restart from the held state with dt / 2^h; the others are held
        std::vector<int> hold(B);
        for (int b = 0; b < B; ++b) {
            hold[b] = retry[b] ? 0 : 1;
            hp[(size_t)RP * b + 3] = retry[b] ? w.hprm[(size_t)RP * b + 3] * (double)(1 << h) : w.hprm[(size_t)RP * b + 3];
        }
        MB_CUDA(cudaMemcpyAsync(w.retry, retry.data(), 4 * B, cudaMemcpyHostToDevice, s));
        MB_CUDA(cudaMemcpyAsync(w.failed, hold.data(), 4 * B, cudaMemcpyHostToDevice, s));
        MB_CUDA(cudaMemcpyAsync(w.prm, hp.data(), 8 * hp.size(), cudaMemcpyHostToDevice, s));
        k_rom_copy<<<nb, 256, 0, s>>>(Nr, B, w.retry, w.a_hold, w.a), count_launch(R->cell);
        MB_CUDA(cudaStreamSynchronize(s));   // the host buffers above go out of scope
        for (int k = 0; k < (1 << h); ++k)
            if ((rc = rom_batch_step(R))) return rc;
        MB_CUDA(cudaMemcpy(f1.data(), w.failed, 4 * B, cudaMemcpyDeviceToHost));
        nretry = 0;
        for (int b = 0; b < B; ++b) {
            retry[b] = retry[b] && f1[b];
            nretry += retry[b];
        }
    }
    // the parameters and the failure flags of every slot back (the held ones as before the step)
    for (int b = 0; b < B; ++b) f1[b] = f0[b] || retry[b];
    MB_CUDA(cudaMemcpyAsync(w.failed, f1.data(), 4 * B, cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemcpyAsync(w.prm, w.hprm.data(), 8 * w.hprm.size(), cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaStreamSynchronize(s));
    return MB_OK;
}
}  // namespace mb

static int rom_solve(mb_rom* R, int B, const mb_rom_params* prm, int n_steps, double dt, double* V_out,
                     double* sac_out, double* a_final, double* a_traj, mb_rom_info* info) {
    const int ncol = n_steps + 1;
    int rc = rom_batch_begin(R, B, prm, dt);
    if (rc) return rc;
    std::vector<double> hV(B), hS(B), ha(a_traj ? (size_t)B * R->d.Nr : 0);
    std::vector<int> hf(B);
    for (int step = 0; step <= n_steps; ++step) {
        if (step > 0 && (rc = rom_step_halving(R, R->cell->opt.max_halvings))) return rc;
        if ((rc = rom_batch_outputs(R, hV.data(), hS.data(), hf.data()))) return rc;
        for (int b = 0; b < B; ++b) {
            V_out[(size_t)b * ncol + step] = hf[b] ? NAN : hV[b];
            sac_out[(size_t)b * ncol + step] = hf[b] ? NAN : hS[b];
        }
        if (a_traj) {
            const int Nr = R->d.Nr;
            MB_CUDA(cudaMemcpy(ha.data(), R->w.a, 8 * ha.size(), cudaMemcpyDeviceToHost));
            for (int b = 0; b < B; ++b)
                memcpy(a_traj + ((size_t)b * ncol + step) * Nr, ha.data() + (size_t)b * Nr, 8 * (size_t)Nr);
        }
    }
    mb_rom_info inf{0, 0, 0};
    for (int b = 0; b < B; ++b) {
        long long its = 0, flips = 0;
        if ((rc = rom_slot_stats(R, b, &its, &flips, a_final ? a_final + (size_t)b * R->d.Nr : nullptr))) return rc;
        inf.newton_its += its;
        inf.flips += flips;
        inf.failed += hf[b] ? 1 : 0;
    }
    if (info) *info = inf;
    if (inf.failed) {
        set_error("mb_rom_solve_batch: reduced Newton did not converge for some instances");
        return MB_ENOCONV;
    }
    return MB_OK;
}

// ------------------------------------------- hierarchical error estimate
// Eq. ap4:estimate with the saturation constant theta of Eq. ap4:saturation:
// per field f (c, phi, plated-Li n) and step, e_f = ||U_f a - Uv_f av||_W /
// (1 - theta), U the reduced model's basis, Uv the validation model's, W the
// L^2 weights of the voxel grid (V per voxel value, A per face value).  With
// Uv W-orthonormal on each field, U_f a = Uv_f (T_f a) + R_f a with R_f a
// W-orthogonal to span Uv_f, so
//   e_f^2 = || T_f a - av|_f ||_2^2 + a^T G_f a,   G_f = R_f^T W R_f,
// T_f and G_f formed once from the bases (no cancellation between the two
// models' reconstructions); per instance and step only O(Nv Nr + Nr^2) flops on
// the coefficients.  One block per instance, FP64, deterministic sums.
namespace mb {

constexpr int EST_THREADS = 256;

__global__ void __launch_bounds__(EST_THREADS)
k_rom_estimate(int Nr, int Nv, const double* __restrict__ a, const double* __restrict__ av,
               const double* __restrict__ T, const int* __restrict__ fld, const double* __restrict__ G, int g0, int g1,
               int g2, const int* __restrict__ failed, const int* __restrict__ failed_v, double scale,
               double* __restrict__ est, double* __restrict__ nrm) {
    __shared__ double sa[ROM_NR_MAX];
    __shared__ double part[EST_THREADS / 32][3];
    __shared__ double npart[EST_THREADS / 32][3];
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < Nr; i += blockDim.x) sa[i] = a[(int64_t)b * Nr + i];
    __syncthreads();
    double acc[3] = {0.0, 0.0, 0.0}, nacc[3] = {0.0, 0.0, 0.0};
    // || T a - av ||^2 per field: one warp per validation mode; and ||av||^2 per
    // field (= ||Uv_f av||_W^2, Uv W-orthonormal on each field)
    for (int j = wid; j < Nv; j += nw) {
        const int f = fld[j];
        if (f < 0) continue;
        double t = 0.0;
        for (int i = lane; i < Nr; i += 32) t = fma(T[(int64_t)j * Nr + i], sa[i], t);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) {
            const double x = av[(int64_t)b * Nv + j];
            const double d = t - x;
            acc[f] = fma(d, d, acc[f]);
            nacc[f] = fma(x, x, nacc[f]);
        }
    }
    // a^T G_f a: one warp per row of G_f
    const int gon[3] = {g0, g1, g2};
    for (int f = 0; f < 3; ++f) {
        if (!gon[f]) continue;
        const double* Gf = G + (int64_t)f * Nr * Nr;
        for (int i = wid; i < Nr; i += nw) {
            double t = 0.0;
            for (int k = lane; k < Nr; k += 32) t = fma(Gf[(int64_t)i * Nr + k], sa[k], t);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) acc[f] = fma(sa[i], t, acc[f]);
        }
    }
    if (lane == 0)
        for (int f = 0; f < 3; ++f) {
            part[wid][f] = acc[f];
            npart[wid][f] = nacc[f];
        }
    __syncthreads();
    if (threadIdx.x < 3) {
        double sum = 0.0, nsum = 0.0;
        for (int w = 0; w < nw; ++w) {
            sum += part[w][threadIdx.x];
            nsum += npart[w][threadIdx.x];
        }
        const bool bad = failed[b] || failed_v[b];
        est[(int64_t)b * 3 + threadIdx.x] = bad ? NAN : scale * sqrt(fmax(sum, 0.0));
        nrm[(int64_t)b * 3 + threadIdx.x] = bad ? NAN : sqrt(nsum);
    }
}


// T, G_f and the fields of the validation modes for the pair (R, Rv)
static int rom_est_setup(mb_rom* R, mb_rom* Rv) {
    RomEst& E = R->est;
    if (E.val == Rv && E.T) return MB_OK;
    for (void* p : E.bufs) cudaFree(p);
    E = RomEst();
    const mb_cell* c = R->cell;
    const int64_t n = c->n, N = c->D.N;
    const int Nr = R->d.Nr, Nv = Rv->d.Nr;
    const std::vector<double>& U = R->hU;
    const std::vector<double>& Uv = Rv->hU;
    const double wv = c->P.V, wa = c->P.A;
    auto wt = [&](int64_t i) { return i < 2 * N ? wv : wa; };
    // field of each validation mode (its nonzero rows must lie in one field)
    std::vector<int> fld(Nv, -1);
    for (int64_t i = 0; i < n; ++i) {
        const int f = est_field(i, N);
        for (int j = 0; j < Nv; ++j)
            if (Uv[(size_t)i * Nv + j] != 0.0) {
                if (fld[j] >= 0 && fld[j] != f) {
                    set_error("mb_rom_estimate_batch: a validation mode spans more than one field");
                    return MB_EINVAL;
                }
                fld[j] = f;
            }
    }
    std::vector<int> vm[3], um[3];   // validation modes of each field; reduced modes nonzero there
    for (int j = 0; j < Nv; ++j)
        if (fld[j] >= 0) vm[fld[j]].push_back(j);
    {
        std::vector<char> seen((size_t)3 * Nr, 0);
        for (int64_t i = 0; i < n; ++i) {
            const int f = est_field(i, N);
            for (int k = 0; k < Nr; ++k)
                if (U[(size_t)i * Nr + k] != 0.0 && !seen[(size_t)f * Nr + k]) {
                    seen[(size_t)f * Nr + k] = 1;
                    um[f].push_back(k);
                }
        }
        for (int f = 0; f < 3; ++f) std::sort(um[f].begin(), um[f].end());
    }
    // Uv must be W-orthonormal on each field
    std::vector<double> Gv((size_t)Nv * Nv, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        const std::vector<int>& V = vm[est_field(i, N)];
        const double w = wt(i);
        for (size_t p = 0; p < V.size(); ++p) {
            const double x = w * Uv[(size_t)i * Nv + V[p]];
            if (x == 0.0) continue;
            for (size_t q = 0; q < V.size(); ++q) Gv[(size_t)V[p] * Nv + V[q]] += x * Uv[(size_t)i * Nv + V[q]];
        }
    }
    for (int f = 0; f < 3; ++f)
        for (int p : vm[f])
            for (int q : vm[f])
                if (fabs(Gv[(size_t)p * Nv + q] - (p == q ? 1.0 : 0.0)) > 1e-8) {
                    set_error("mb_rom_estimate_batch: the validation basis is not W-orthonormal on each field");
                    return MB_EINVAL;
                }
    // T[j][k] = sum over rows of field f(j) of w Uv[., j] U[., k]
    std::vector<double> T((size_t)Nv * Nr, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        const int f = est_field(i, N);
        const double w = wt(i);
        for (int j : vm[f]) {
            const double x = w * Uv[(size_t)i * Nv + j];
            if (x == 0.0) continue;
            for (int k : um[f]) T[(size_t)j * Nr + k] += x * U[(size_t)i * Nr + k];
        }
    }
    // G_f = sum over rows of field f of w r r^T, r = U row - Uv row T (only the modes nonzero there)
    std::vector<double> G((size_t)3 * Nr * Nr, 0.0);
    std::vector<double> r(Nr);
    for (int64_t i = 0; i < n; ++i) {
        const int f = est_field(i, N);
        if (um[f].empty()) continue;
        const double w = wt(i);
        for (int k : um[f]) {
            double x = U[(size_t)i * Nr + k];
            for (int j : vm[f]) x -= Uv[(size_t)i * Nv + j] * T[(size_t)j * Nr + k];
            r[k] = x;
        }
        double* Gf = G.data() + (size_t)f * Nr * Nr;
        for (int k : um[f]) {
            const double x = w * r[k];
            if (x == 0.0) continue;
            for (int l : um[f]) Gf[(size_t)k * Nr + l] += x * r[l];
        }
    }
    for (int f = 0; f < 3; ++f)
        for (size_t q = 0; q < (size_t)Nr * Nr && !E.gon[f]; ++q) E.gon[f] = G[(size_t)f * Nr * Nr + q] != 0.0;
    E.T = rom_alloc<double>(E.bufs, T.size());
    E.G = rom_alloc<double>(E.bufs, G.size());
    E.fld = rom_alloc<int>(E.bufs, Nv);
    if (!E.T || !E.G || !E.fld) return MB_ENOMEM;
    MB_CUDA(cudaMemcpy(E.T, T.data(), 8 * T.size(), cudaMemcpyHostToDevice));
    MB_CUDA(cudaMemcpy(E.G, G.data(), 8 * G.size(), cudaMemcpyHostToDevice));
    MB_CUDA(cudaMemcpy(E.fld, fld.data(), 4 * fld.size(), cudaMemcpyHostToDevice));
    E.val = Rv;
    E.Nv = Nv;
    return MB_OK;
}

}  // namespace mb

extern "C" int mb_rom_estimate_batch(mb_rom* R, mb_rom* Rv, double theta, int B, const mb_rom_params* prm,
                                     int n_steps, double dt, double* V_out, double* Vv_out, double* est_out,
                                     double* norm_out, mb_rom_info* info) {
    if (!R || !Rv || R == Rv || !(theta >= 0.0 && theta < 1.0) || B < 1 || !prm || n_steps < 0 || !(dt > 0) ||
        !est_out) {
        set_error("mb_rom_estimate_batch: invalid argument");
        return MB_EINVAL;
    }
    if (R->cell->n != Rv->cell->n || R->cell->D.N != Rv->cell->D.N) {
        set_error("mb_rom_estimate_batch: the two models belong to cells of different sizes");
        return MB_EINVAL;
    }
    int rc = rom_est_setup(R, Rv);
    if (rc) return rc;
    RomEst& E = R->est;
    if (E.Bcap < B) {
        E.est = rom_alloc<double>(E.bufs, (size_t)3 * B);
        E.nrm = rom_alloc<double>(E.bufs, (size_t)3 * B);
        if (!E.est || !E.nrm) { set_error("mb_rom_estimate_batch: device memory"); return MB_ENOMEM; }
        E.Bcap = B;
    }
    if ((rc = rom_batch_begin(R, B, prm, dt)) || (rc = rom_batch_begin(Rv, B, prm, dt))) return rc;
    const int ncol = n_steps + 1;
    const double scale = 1.0 / (1.0 - theta);
    std::vector<double> hV(B), hS(B), hVv(B), hSv(B), he((size_t)3 * B), hn((size_t)3 * B);
    std::vector<int> hf(B), hfv(B);
    cudaStream_t s = R->cell->stream;
    for (int step = 0; step <= n_steps; ++step) {
        if (step > 0 && ((rc = rom_step_halving(R, R->cell->opt.max_halvings)) ||
                         (rc = rom_step_halving(Rv, Rv->cell->opt.max_halvings))))
            return rc;
        // both streams are idle after their outputs are read
        if ((rc = rom_batch_outputs(R, hV.data(), hS.data(), hf.data())) ||
            (rc = rom_batch_outputs(Rv, hVv.data(), hSv.data(), hfv.data())))
            return rc;
        k_rom_estimate<<<(unsigned)B, EST_THREADS, 0, s>>>(R->d.Nr, E.Nv, R->w.a, Rv->w.a, E.T, E.fld, E.G, E.gon[0],
                                                          E.gon[1], E.gon[2], R->w.failed, Rv->w.failed, scale,
                                                          E.est, E.nrm), count_launch(R->cell);
        MB_CUDA_LAUNCH("rom_estimate");
        MB_CUDA(cudaMemcpyAsync(he.data(), E.est, 8 * he.size(), cudaMemcpyDeviceToHost, s));
        MB_CUDA(cudaMemcpyAsync(hn.data(), E.nrm, 8 * hn.size(), cudaMemcpyDeviceToHost, s));
        MB_CUDA(cudaStreamSynchronize(s));
        for (int b = 0; b < B; ++b) {
            for (int f = 0; f < 3; ++f) {
                est_out[((size_t)b * ncol + step) * 3 + f] = he[(size_t)b * 3 + f];
                if (norm_out) norm_out[((size_t)b * ncol + step) * 3 + f] = hn[(size_t)b * 3 + f];
            }
            if (V_out) V_out[(size_t)b * ncol + step] = hf[b] ? NAN : hV[b];
            if (Vv_out) Vv_out[(size_t)b * ncol + step] = hfv[b] ? NAN : hVv[b];
        }
    }
    mb_rom_info inf{0, 0, 0};
    for (int b = 0; b < B; ++b) {
        long long its = 0, flips = 0;
        if ((rc = rom_slot_stats(R, b, &its, &flips, nullptr))) return rc;
        inf.newton_its += its;
        inf.flips += flips;
        inf.failed += (hf[b] || hfv[b]) ? 1 : 0;
    }
    if (info) *info = inf;
    if (inf.failed) {
        set_error("mb_rom_estimate_batch: reduced Newton did not converge for some instances");
        return MB_ENOCONV;
    }
    return MB_OK;
}

// ------------------------------------------------------------ test hooks
#include "../../include/mb_debug.h"

extern "C" int mb_debug_rom_jac(int Nr, int M, int B, const float* P, const float* GU, const float* Ms,
                                const float* Alin, const double* dt_inv, int tc, float* J) {
    if (Nr < 1 || M < 1 || B < 1 || !P || !GU || !Ms || !Alin || !dt_inv || !J) {
        set_error("mb_debug_rom_jac: invalid argument");
        return MB_EINVAL;
    }
    std::vector<void*> bufs;
    RomDev d;
    d.Nr = Nr;
    d.M = M;
    d.tc = tc;
    auto dev = [&](const void* h, size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes ? bytes : 1) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        if (h && cudaMemcpy(p, h, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
        return p;
    };
    std::vector<double> prm((size_t)RP * B, 0.0);
    for (int b = 0; b < B; ++b) prm[(size_t)RP * b + 3] = dt_inv[b];
    std::vector<int> hp(B, 0);
    std::vector<float> Pt((size_t)M * Nr);
    for (int i = 0; i < Nr; ++i)
        for (int k = 0; k < M; ++k) Pt[(size_t)k * Nr + i] = P[(size_t)i * M + k];
    d.Ptf = (float*)dev(Pt.data(), 4 * Pt.size());
    d.Msf = (float*)dev(Ms, 4 * (size_t)Nr * Nr);
    d.Alinf = (float*)dev(Alin, 4 * (size_t)Nr * Nr);
    float* gu = (float*)dev(GU, 4 * (size_t)M * B * Nr);
    double* dprm = (double*)dev(prm.data(), 8 * prm.size());
    int* dhp = (int*)dev(hp.data(), 4 * (size_t)B);
    float* dJ = (float*)dev(nullptr, 4 * (size_t)B * Nr * Nr);
    int rc = MB_OK;
    if (!d.Ptf || !d.Msf || !d.Alinf || !gu || !dprm || !dhp || !dJ) {
        rc = cuda_fail(cudaGetLastError(), "debug_rom_jac alloc");
    } else {
        const dim3 gj((unsigned)(((int64_t)B * Nr + JT_COLS - 1) / JT_COLS), (unsigned)((Nr + JT_ROWS - 1) / JT_ROWS));
        int* derr = (int*)dev(nullptr, 16);
        if (derr) cudaMemset(derr, 0, 16);
        if (tc == 2) {
            if (!derr || !t5_prepare(d, bufs)) {
                set_error("debug_rom_jac: the tcgen05 GEMM cannot run this size");
                rc = MB_EINVAL;
            } else {
                k_rom_jac5<<<(unsigned)(((int64_t)B * Nr + T5_M - 1) / T5_M), T5_THREADS, T5_SMEM>>>(
                    d, B, B, nullptr, dprm, gu, dhp, dJ, nullptr, nullptr, derr);
            }
        } else if (tc) {
            k_rom_jac<true><<<gj, 256>>>(d, B, B, nullptr, dprm, gu, dhp, dJ, nullptr, nullptr);
        } else {
            k_rom_jac<false><<<gj, 256>>>(d, B, B, nullptr, dprm, gu, dhp, dJ, nullptr, nullptr);
        }
        if (!rc) {
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpy(J, dJ, 4 * (size_t)B * Nr * Nr, cudaMemcpyDeviceToHost);
            int herr = 0;
            if (e == cudaSuccess && derr) e = cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) rc = cuda_fail(e, "debug_rom_jac");
            else if (herr) { set_error("debug_rom_jac: a bounded wait of the tcgen05 GEMM gave up"); rc = MB_ETIMEOUT; }
        }
    }
    for (void* p : bufs) cudaFree(p);
    return rc;
}

template <class T>
static int debug_rom_lu(int Nr, int B, int in_place, const double* J, const double* r, double* delta) {
    const bool smem = !in_place;
    if (smem && lu_smem(Nr, sizeof(T)) > ROM_LU_SMEM) {
        set_error("mb_debug_rom_lu: matrix too large for shared memory");
        return MB_EINVAL;
    }
    std::vector<T> hJ(J, J + (size_t)B * Nr * Nr);
    std::vector<int> ones(B, 1), zeros(B, 0);
    T* dJ = nullptr;
    double *dr = nullptr, *dd = nullptr;
    int *da = nullptr, *dh = nullptr;
    cudaError_t e = cudaMalloc(&dJ, sizeof(T) * hJ.size());
    if (e == cudaSuccess) e = cudaMalloc(&dr, 8 * (size_t)B * Nr);
    if (e == cudaSuccess) e = cudaMalloc(&dd, 8 * (size_t)B * Nr);
    if (e == cudaSuccess) e = cudaMalloc(&da, 4 * (size_t)B);
    if (e == cudaSuccess) e = cudaMalloc(&dh, 4 * (size_t)B);
    if (e == cudaSuccess) e = cudaMemcpy(dJ, hJ.data(), sizeof(T) * hJ.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dr, r, 8 * (size_t)B * Nr, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(da, ones.data(), 4 * (size_t)B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dh, zeros.data(), 4 * (size_t)B, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(smem ? k_rom_lu<T, true> : k_rom_lu<T, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ROM_LU_SMEM);
    if (e == cudaSuccess) {
        const unsigned lt = Nr <= 96 ? LU_T_SMALL : LU_T_LARGE;
        if (smem)
            k_rom_lu<T, true><<<(unsigned)B, lt, lu_smem(Nr, sizeof(T))>>>(Nr, dJ, dr, da, dh, 0, nullptr, dd);
        else
            k_rom_lu<T, false><<<(unsigned)B, lt, ROM_LU_SMEM>>>(Nr, dJ, dr, da, dh, 0, nullptr, dd);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(delta, dd, 8 * (size_t)B * Nr, cudaMemcpyDeviceToHost);
    cudaFree(dJ);
    cudaFree(dr);
    cudaFree(dd);
    cudaFree(da);
    cudaFree(dh);
    return e == cudaSuccess ? MB_OK : cuda_fail(e, "debug_rom_lu");
}

extern "C" int mb_debug_rom_lu(int Nr, int B, int fp64, int in_place, const double* J, const double* r,
                               double* delta) {
    if (Nr < 1 || Nr > ROM_NR_MAX || B < 1 || !J || !r || !delta) {
        set_error("mb_debug_rom_lu: invalid argument");
        return MB_EINVAL;
    }
    return fp64 ? debug_rom_lu<double>(Nr, B, in_place, J, r, delta)
                : debug_rom_lu<float>(Nr, B, in_place, J, r, delta);
}

extern "C" int mb_debug_rom_refine(mb_rom* R, int on) {
    if (!R) return MB_EINVAL;
    R->d.ir = on ? 1 : 0;
    return MB_OK;
}

extern "C" int mb_debug_rom_graph(mb_rom* R, int on) {
    if (!R) return MB_EINVAL;
    R->d.graph = on ? 1 : 0;
    return MB_OK;
}

extern "C" int mb_debug_rom_tensor(mb_rom* R, int on) {
    if (!R || on < 0 || on > 2) return MB_EINVAL;
    if (on == 2 && !R->d.Pbf) {
        set_error("mb_debug_rom_tensor: the tcgen05 GEMM does not take this model (N_r > 256)");
        return MB_EINVAL;
    }
    R->d.tc = on;
    R->tc_forced = true;
    return MB_OK;
}

extern "C" int mb_debug_rom_slot(mb_rom* R, int b, int* failed, int* pass_its, float* last_norm, int* escalated) {
    if (!R || b < 0 || b >= R->w.B || !failed || !pass_its || !last_norm || !escalated) {
        set_error("mb_debug_rom_slot: invalid argument");
        return MB_EINVAL;
    }
    const RomWork& w = R->w;
    if (cudaMemcpy(failed, w.failed + b, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(pass_its, w.pit + b, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(last_norm, w.dnprev + b, 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(escalated, w.hp + b, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "mb_debug_rom_slot");
    return MB_OK;
}

extern "C" int mb_debug_rom_gemm_tuning(mb_rom* R, int* choice, float* ms) {
    if (!R || !choice || !ms) { set_error("mb_debug_rom_gemm_tuning: invalid argument"); return MB_EINVAL; }
    *choice = R->d.tc;
    for (int k = 0; k < 3; ++k) ms[k] = R->tune_ms[k];
    return MB_OK;
}
