// fom.cu -- full-order kernels: geometry ingest and face classification,
// fused residual, analytic Jacobian-vector product, rest state, plating gates,
// reductions (norms, functionals).
#include <cuda_runtime.h>
#include <stdio.h>

#include "mb_internal.h"
#include "mb_reduce.cuh"

namespace mb {

// ------------------------------------------------------------------ helpers
__device__ inline void vox_coords(const Dims& D, int& z, int& y, int& t) {
    z = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y * blockDim.y + threadIdx.y;
    t = blockIdx.z;
}

static inline dim3 vox_grid(const Dims& D, dim3 blk) {
    return dim3((D.nz + blk.x - 1) / blk.x, (D.ny + blk.y - 1) / blk.y, D.nt);
}
static const dim3 VOX_BLOCK(32, 8, 1);

__device__ inline bool forbidden_pair(int a, int b) {
    auto f = [](int x, int y) {
        return (x == PG && y == PK) || (x == PG && y == PCP) || (x == PK && y == PCN) ||
               (x == PCN && y == PCP) || (x == PK && y == PL);
    };
    return f(a, b) || f(b, a);
}

// --------------------------------------------------- K0: face classification
// Pass 1: per voxel, mask of electrolyte neighbours of graphite voxels and the
// number of plating faces it owns; flags forbidden contacts.
__global__ void k_classify_count(Dims D, const uint8_t* __restrict__ lab, uint8_t* __restrict__ emask,
                                 uint32_t* __restrict__ cnt, int* __restrict__ err) {
    int z, y, t;
    vox_coords(D, z, y, t);
    if (z >= D.nz || y >= D.ny) return;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    int lv = lab[v];
    if (lv > 5) { atomicOr(err, 2); }
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
    uint32_t m = 0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (!inb[d]) continue;
        int lw = lab[v + off[d]];
        if (forbidden_pair(lv, lw)) atomicOr(err, 1);
        if (lv == PG && lw == PE) m |= 1u << d;
        // collector contacts with electrode solid (bit 2: CN, bit 3: CP)
        if (lv == PCN && (lw == PG || lw == PL)) atomicOr(err, 4);
        if (lv == PCP && (lw == PK || lw == PL)) atomicOr(err, 8);
    }
    emask[v] = (uint8_t)m;
    cnt[v] = __popc(m);
}

// Exclusive scan of uint32 counts (three kernels: block scans, scan of block
// sums in one block, add-back).  SCAN_B elements per block.
constexpr int SCAN_T = 512;
constexpr int SCAN_B = 2 * SCAN_T;

__global__ void k_scan_blocks(const uint32_t* __restrict__ in, int64_t n, uint32_t* __restrict__ out,
                              uint32_t* __restrict__ bsum) {
    __shared__ uint32_t s[SCAN_B];
    int64_t base = (int64_t)blockIdx.x * SCAN_B;
    for (int i = threadIdx.x; i < SCAN_B; i += SCAN_T) s[i] = (base + i < n) ? in[base + i] : 0u;
    __syncthreads();
    // Hillis-Steele inclusive scan in shared memory (simple, done once per cell)
    for (int off = 1; off < SCAN_B; off <<= 1) {
        uint32_t a[2];
        for (int k = 0; k < 2; ++k) {
            int i = threadIdx.x + k * SCAN_T;
            a[k] = (i >= off) ? s[i - off] : 0u;
        }
        __syncthreads();
        for (int k = 0; k < 2; ++k) s[threadIdx.x + k * SCAN_T] += a[k];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < SCAN_B; i += SCAN_T)
        if (base + i < n) out[base + i] = (i == 0 ? 0u : s[i - 1]);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s[SCAN_B - 1];
}

__global__ void k_scan_sums(uint32_t* bsum, int64_t nb, uint32_t* total) {
    // single block: sequential chunks per thread then a shared-memory scan
    __shared__ uint32_t part[1024];
    int64_t per = (nb + blockDim.x - 1) / blockDim.x;
    int64_t b0 = threadIdx.x * per;
    int64_t b1 = b0 + per < nb ? b0 + per : nb;
    uint32_t acc = 0;
    for (int64_t i = b0; i < b1; ++i) acc += bsum[i];
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) { uint32_t x = part[i]; part[i] = run; run += x; }
        *total = run;
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (int64_t i = b0; i < b1; ++i) { uint32_t x = bsum[i]; bsum[i] = run; run += x; }
}

__global__ void k_scan_add(uint32_t* out, int64_t n, const uint32_t* bsum) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / SCAN_B];
}

// Pass 2: per-voxel code and the plating face list.
__global__ void k_classify_write(Dims D, const uint8_t* __restrict__ lab, const uint8_t* __restrict__ emask,
                                 const uint32_t* __restrict__ fbase, uint32_t* __restrict__ vcode,
                                 int32_t* __restrict__ pf_g, int32_t* __restrict__ pf_e,
                                 int8_t* __restrict__ pf_dir) {
    int z, y, t;
    vox_coords(D, z, y, t);
    if (z >= D.nz || y >= D.ny) return;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    uint32_t m = emask[v];
    uint32_t fb = fbase[v];
    vcode[v] = (uint32_t)lab[v] | (m << 3) | (fb << VC_FBASE_SHIFT);
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    uint32_t f = fb;
    for (int d = 0; d < 6; ++d) {
        if (m & (1u << d)) {
            pf_g[f] = (int32_t)v;
            pf_e[f] = (int32_t)(v + off[d]);
            pf_dir[f] = (int8_t)d;
            ++f;
        }
    }
}

int launch_classify(mb_cell* c, const uint8_t* d_lab) {
    const Dims& D = c->D;
    cudaStream_t s = c->stream;
    int64_t N = D.N;
    int64_t nb = (N + SCAN_B - 1) / SCAN_B;
    uint8_t* emask = nullptr;
    uint32_t *cnt = nullptr, *fbase = nullptr, *bsum = nullptr, *total = nullptr;
    int* err = nullptr;
    MB_CUDA(cudaMalloc(&emask, N));
    MB_CUDA(cudaMalloc(&cnt, N * 4));
    MB_CUDA(cudaMalloc(&fbase, N * 4));
    MB_CUDA(cudaMalloc(&bsum, nb * 4 + 16));
    MB_CUDA(cudaMalloc(&total, 16));
    MB_CUDA(cudaMalloc(&err, 16));
    MB_CUDA(cudaMemsetAsync(err, 0, 4, s));
    k_classify_count<<<vox_grid(D, VOX_BLOCK), VOX_BLOCK, 0, s>>>(D, d_lab, emask, cnt, err), ::mb::count_launch(c);
    k_scan_blocks<<<(unsigned)nb, SCAN_T, 0, s>>>(cnt, N, fbase, bsum), ::mb::count_launch(c);
    k_scan_sums<<<1, 1024, 0, s>>>(bsum, nb, total), ::mb::count_launch(c);
    k_scan_add<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(fbase, N, bsum), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("classify");
    int h_err = 0;
    uint32_t h_total = 0;
    MB_CUDA(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaMemcpyAsync(&h_total, total, 4, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    int rc = MB_OK;
    if (h_err & 2) {
        set_error("labels must be in 0..5");
        rc = MB_EINVAL;
    } else if (h_err & 1) {
        set_error("forbidden phase contact (G-K, G-CP, K-CN, K-L or CN-CP)");
        rc = MB_EBADGEOM;
    } else if ((c->count[PCN] > 0 && !(h_err & 4)) || (c->count[PCP] > 0 && !(h_err & 8))) {
        set_error("a current collector touches no electrode solid (its potential would float)");
        rc = MB_EBADGEOM;
    } else if (h_total >= VC_MAX_FACES) {
        set_error("too many plating faces for the 23-bit face index");
        rc = MB_EINVAL;
    }
    if (rc == MB_OK) {
        c->D.F = h_total;
        c->n = 2 * N + (int64_t)h_total;
        size_t F = h_total ? h_total : 1;
        c->vcode = (uint32_t*)cell_alloc(c, N * 4);
        c->pf_g = (int32_t*)cell_alloc(c, F * 4);
        c->pf_e = (int32_t*)cell_alloc(c, F * 4);
        c->pf_dir = (int8_t*)cell_alloc(c, F);
        if (!c->vcode || !c->pf_g || !c->pf_e || !c->pf_dir) rc = MB_ENOMEM;
    }
    if (rc == MB_OK) {
        k_classify_write<<<vox_grid(D, VOX_BLOCK), VOX_BLOCK, 0, s>>>(
            c->D, d_lab, emask, fbase, c->vcode, c->pf_g, c->pf_e, c->pf_dir), ::mb::count_launch(c);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "classify_write");
    }
    cudaStreamSynchronize(s);
    cudaFree(emask); cudaFree(cnt); cudaFree(fbase); cudaFree(bsum); cudaFree(total); cudaFree(err);
    return rc;
}

// ------------------------------------------------------------ rest state
__global__ void k_init_state(DevParams P, Dims D, const uint32_t* __restrict__ vc, double xg, double xk,
                             double cE, double cmaxG, double cmaxK, int hasK, double* __restrict__ u) {
    int z, y, t;
    vox_coords(D, z, y, t);
    if (z >= D.nz || y >= D.ny) return;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    int l = vc_phase(vc[v]);
    double cg = xg * cmaxG, ck = xk * cmaxK;
    double phiE = -ocp_val<double>(P.ocpG, cg / cmaxG);
    double phiK = phiE + ocp_val<double>(P.ocpK, ck / cmaxK);
    double c = 0.0, ph = 0.0;
    switch (l) {
        case PE: c = cE; ph = phiE; break;
        case PG: c = cg; ph = 0.0; break;
        case PK: c = ck; ph = phiK; break;
        case PL: ph = phiE; break;
        case PCN: ph = 0.0; break;
        case PCP: ph = hasK ? phiK : phiE; break;
    }
    u[v] = c;
    u[D.N + v] = ph;
}

int launch_init_state(mb_cell* c, double* u) {
    const Dims& D = c->D;
    if (D.F) MB_CUDA(cudaMemsetAsync(u + 2 * D.N, 0, D.F * 8, c->stream));
    k_init_state<<<vox_grid(D, VOX_BLOCK), VOX_BLOCK, 0, c->stream>>>(
        c->P, D, c->vcode, c->prm.G_x0, c->prm.K_x0, c->prm.E_c0, c->prm.G_cmax, c->prm.K_cmax,
        c->count[PK] > 0 ? 1 : 0, u), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("init_state");
    return MB_OK;
}

// ------------------------------------------------------------ K1: residual
// One thread per voxel; R_c, R_phi of the voxel from its storage term, its six
// face fluxes (bulk, conduction, interface kinetics with plating) and the
// outer-boundary terms; a graphite voxel also writes the rows R_n of its
// plating faces.
template <class T>
__global__ void __launch_bounds__(256)
k_residual(DevParams P, Dims D, const uint32_t* __restrict__ vc, const T* __restrict__ u,
           const double* __restrict__ uold, const uint8_t* __restrict__ gate, double dt_inv,
           double I_app, double s_i0d, double k_pld, T* __restrict__ r) {
    int z, y, t;
    vox_coords(D, z, y, t);
    if (z >= D.nz || y >= D.ny) return;
    const int64_t N = D.N;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    const T* __restrict__ cc = u;
    const T* __restrict__ ph = u + N;
    const T* __restrict__ nn = u + 2 * N;
    const T s_i0 = T(s_i0d), k_pl = T(k_pld);
    uint32_t code = vc[v];
    int lv = vc_phase(code);
    T cv = cc[v], pv = ph[v];
    T rc = T(0), rp = T(0);
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
    uint32_t fb = vc_fbase(code);
    int rank = 0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (!inb[d]) continue;
        int64_t w = v + off[d];
        uint32_t cw_code = vc[w];
        int lw = vc_phase(cw_code);
        T cw = cc[w], pw = ph[w];
        T nf = T(0);
        bool g = false;
        int64_t f = -1;
        if (lv == PG && lw == PE) {
            f = fb + rank;
            ++rank;
        } else if (lv == PE && lw == PG) {
            uint32_t emw = vc_emask(cw_code);
            f = vc_fbase(cw_code) + __popc(emw & ((1u << opp_dir(d)) - 1u));
        }
        if (f >= 0) {
            nf = nn[f];
            g = gate[f] != 0;
        }
        T ipl = T(0);
        face_residual<T>(P, lv, lw, cv, pv, cw, pw, nf, g, s_i0, k_pl, rc, rp, ipl);
        if (lv == PG && lw == PE)
            r[2 * N + f] = (nf - T(uold[2 * N + f])) * T(dt_inv) + ipl * T(P.invF);
    }
    if (t == 0 && lv == PCN) rp += T(P.g_dir) * pv;
    if (t == D.nt - 1 && lv == PCP) rp += T(P.A) * T(I_app);
    if (has_c(lv)) rc += T(P.V) * (cv - T(uold[v])) * T(dt_inv);
    else rc = cv;
    r[v] = rc;
    r[N + v] = rp;
}

template <class T>
int launch_residual(mb_cell* c, const T* u, const double* u_old, const uint8_t* gate, double dt,
                    double I_app, T* r, cudaStream_t s) {
    const Dims& D = c->D;
    cudaEvent_t ev;
    prof_begin(c, s, &ev);
    k_residual<T><<<vox_grid(D, VOX_BLOCK), VOX_BLOCK, 0, s>>>(c->P, D, c->vcode, u, u_old, gate,
                                                               1.0 / dt, I_app, c->s_i0, c->k_pl, r), ::mb::count_launch(c);
    prof_end(c, s, PROF_RESIDUAL, ev);
    MB_CUDA_LAUNCH("residual");
    return MB_OK;
}
template int launch_residual<double>(mb_cell*, const double*, const double*, const uint8_t*, double,
                                     double, double*, cudaStream_t);
template int launch_residual<float>(mb_cell*, const float*, const double*, const uint8_t*, double,
                                    double, float*, cudaStream_t);

// ------------------------------------------------------------ K2: JVP
// J(u) v from the analytic per-face partial derivatives (chain rule through
// sqrt, sinh, cosh, exp, 1/cbar, U0'(c) and f_pre'(n)).
// With SCALED, x is in scaled unknowns (x_hat = x / s_u) and each output row
// is divided by the residual scale s_r and by the magnitude of its own
// diagonal entry in these units: the Krylov operator E S_r^-1 J S_u with
// E = |diag(S_r^-1 J S_u)|^-1, so that every row of the Krylov system has a
// unit diagonal whatever its physical scale (collector and electrolyte rows
// differ by ~1e10 otherwise).
// TC: precision of the linearisation point and of the nonlinear per-face
// coefficients; TV: precision of the direction x, of its differences and of
// the result.  (TC, TV) = (double, double) is the FP64 operator, (float,
// double) the mixed one (FP32 transcendentals/divisions, FP64 vectors), and
// (float, float) the all-FP32 variant of the C-ABI.
template <class TC, class TV, int MODE>
__global__ void __launch_bounds__(256)
k_jvp(DevParams P, Dims D, const uint32_t* __restrict__ vc, const TC* __restrict__ u,
      const uint8_t* __restrict__ gate, double dt_inv, double s_i0d, double k_pld,
      const TV* __restrict__ x, TV* __restrict__ y_out) {
    int z, y, t;
    vox_coords(D, z, y, t);
    if (z >= D.nz || y >= D.ny) return;
    constexpr bool SCALED = MODE >= 1, EQUIL = MODE == 2;
    const int64_t N = D.N;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    const TC* __restrict__ cc = u;
    const TC* __restrict__ ph = u + N;
    const TC* __restrict__ nn = u + 2 * N;
    const TC s_i0 = TC(s_i0d), k_pl = TC(k_pld);
    uint32_t code = vc[v];
    int lv = vc_phase(code);
    TC cv = cc[v], pv = ph[v];
    const TV nc = TV(sqrt(sqrt(P.nc4)));
    const TV idt = TV(dt_inv);
    TV dcv = x[v], dpv = x[N + v];
    if (SCALED) dcv *= TV(P.cref[lv]);
    TV jc = TV(0), jp = TV(0);
    TV dgc = TV(0), dgp = TV(0);   // diagonal entries d R_c(v)/d c_v, d R_phi(v)/d phi_v
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
    uint32_t fb = vc_fbase(code);
    int rank = 0;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (!inb[d]) continue;
        int64_t w = v + off[d];
        uint32_t cw_code = vc[w];
        int lw = vc_phase(cw_code);
        TC cw = cc[w], pw = ph[w];
        TV dcw = x[w], dpw = x[N + w];
        if (SCALED) dcw *= TV(P.cref[lw]);
        TC nf = TC(0);
        TV dnf = TV(0);
        bool g = false;
        int64_t f = -1;
        if (lv == PG && lw == PE) {
            f = fb + rank;
            ++rank;
        } else if (lv == PE && lw == PG) {
            uint32_t emw = vc_emask(cw_code);
            f = vc_fbase(cw_code) + __popc(emw & ((1u << opp_dir(d)) - 1u));
        }
        if (f >= 0) {
            nf = nn[f];
            dnf = x[2 * N + f];
            if (SCALED) dnf *= nc;
            g = gate[f] != 0;
        }
        TV jn = TV(0), jnn = TV(0);
        face_jvp<TC, TV>(P, lv, lw, cv, pv, cw, pw, nf, g, s_i0, k_pl, dcv, dpv, dcw, dpw, dnf, jc, jp, jn, jnn,
                         dgc, dgp);
        if (lv == PG && lw == PE) {
            jn += dnf * idt;
            if (SCALED) jn *= TV(1) / (nc * idt);
            if (EQUIL) jn *= TV(1) / fabs(TV(1) + jnn / idt);
            y_out[2 * N + f] = jn;
        }
    }
    if (t == 0 && lv == PCN) {
        jp += TV(P.g_dir) * dpv;
        dgp += TV(P.g_dir);
    }
    const TV Vdt = TV(P.V * dt_inv);
    if (has_c(lv)) {
        jc += Vdt * dcv;
        dgc += Vdt;
    } else {
        jc = dcv;
    }
    if (SCALED && !EQUIL) {
        jc *= has_c(lv) ? TV(1) / (Vdt * TV(P.cref[lv])) : TV(1);
        jp *= TV(1) / TV(P.A);
    }
    if (EQUIL) {
        // row c: s_r = V c_ref/dt, diagonal dgc * c_ref / s_r = dgc dt / V; row phi: s_r = A, diagonal dgp / A
        if (has_c(lv)) jc *= TV(1) / (Vdt * TV(P.cref[lv]) * tmax(fabs(dgc / Vdt), TV(1e-30)));
        jp *= TV(1) / tmax(fabs(dgp), TV(1e-30) * TV(P.A));
    }
    y_out[v] = jc;
    y_out[N + v] = jp;
}

template <class TC, class TV>
int launch_jvp(mb_cell* c, const TC* u, const uint8_t* gate, double dt, const TV* v, TV* jv, cudaStream_t s,
               int mode) {
    const Dims& D = c->D;
    const dim3 g = vox_grid(D, VOX_BLOCK);
    cudaEvent_t ev;
    prof_begin(c, s, &ev);
    if (mode == 2)
        k_jvp<TC, TV, 2><<<g, VOX_BLOCK, 0, s>>>(c->P, D, c->vcode, u, gate, 1.0 / dt, c->s_i0, c->k_pl, v, jv), ::mb::count_launch(c);
    else if (mode == 1)
        k_jvp<TC, TV, 1><<<g, VOX_BLOCK, 0, s>>>(c->P, D, c->vcode, u, gate, 1.0 / dt, c->s_i0, c->k_pl, v, jv), ::mb::count_launch(c);
    else
        k_jvp<TC, TV, 0><<<g, VOX_BLOCK, 0, s>>>(c->P, D, c->vcode, u, gate, 1.0 / dt, c->s_i0, c->k_pl, v, jv), ::mb::count_launch(c);
    prof_end(c, s, PROF_JVP, ev);
    MB_CUDA_LAUNCH("jvp");
    return MB_OK;
}
template int launch_jvp<double, double>(mb_cell*, const double*, const uint8_t*, double, const double*, double*,
                                        cudaStream_t, int);
template int launch_jvp<float, double>(mb_cell*, const float*, const uint8_t*, double, const double*, double*,
                                       cudaStream_t, int);
template int launch_jvp<float, float>(mb_cell*, const float*, const uint8_t*, double, const float*, float*,
                                      cudaStream_t, int);

// ------------------------------------------------------------ plating gates
__global__ void k_gate(Dims D, const int32_t* __restrict__ pg, const int32_t* __restrict__ pe,
                       const double* __restrict__ u, const double* __restrict__ n_old,
                       uint8_t* __restrict__ gate) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= D.F) return;
    const double* ph = u + D.N;
    double etap = ph[pg[f]] - ph[pe[f]];
    gate[f] = (n_old[f] > 0.0 || etap < 0.0) ? 1 : 0;
}

int launch_gate(mb_cell* c, const double* u, const double* n_old, uint8_t* gate, cudaStream_t s) {
    if (c->D.F == 0) return MB_OK;
    k_gate<<<(unsigned)((c->D.F + 255) / 256), 256, 0, s>>>(c->D, c->pf_g, c->pf_e, u, n_old, gate), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("gate");
    return MB_OK;
}

int launch_gate_residual_unprofiled(mb_cell* c, const double* u, const double* u_old, uint8_t* gate_scratch,
                                    double dt, double I_app, double* r, cudaStream_t s) {
    const Dims& D = c->D;
    if (D.F > 0) {
        k_gate<<<(unsigned)((D.F + 255) / 256), 256, 0, s>>>(D, c->pf_g, c->pf_e, u_old, u_old + 2 * D.N,
                                                             gate_scratch), ::mb::count_launch(c);
        MB_CUDA_LAUNCH("gate");
    }
    k_residual<double><<<vox_grid(D, VOX_BLOCK), VOX_BLOCK, 0, s>>>(c->P, D, c->vcode, u, u_old, gate_scratch,
                                                                    1.0 / dt, I_app, c->s_i0, c->k_pl, r),
        ::mb::count_launch(c);
    MB_CUDA_LAUNCH("residual");
    return MB_OK;
}

// ------------------------------------------------------------ reductions
// Deterministic reductions (mb_reduce.cuh).
__global__ void __launch_bounds__(RED_THREADS)
k_scaled_max(DevParams P, Dims D, const uint32_t* __restrict__ vc, const double* __restrict__ x,
             int which, double dt_inv, double* partials) {
    double acc[1] = {0.0};
    int64_t n = 2 * D.N + D.F;
    double nc = sqrt(sqrt(P.nc4));
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s;
        if (i < D.N) {
            int l = vc_phase(vc[i]);
            s = which == 0 ? P.cref[l] : (has_c(l) ? P.V * P.cref[l] * dt_inv : 1.0);
        } else if (i < 2 * D.N) {
            s = which == 0 ? 1.0 : P.A;
        } else {
            s = which == 0 ? nc : nc * dt_inv;
        }
        double a = fabs(x[i]) / s;
        if (!(a == a)) a = 1e300;   // NaN -> huge
        acc[0] = fmax(acc[0], a);
    }
    block_reduce_store<1, true>(acc, partials);
}

int scaled_maxnorm(mb_cell* c, const double* x, int which, double dt, double* out) {
    cudaStream_t s = c->stream;
    k_scaled_max<<<RED_BLOCKS, RED_THREADS, 0, s>>>(c->P, c->D, c->vcode, x, which, 1.0 / dt, c->red), ::mb::count_launch(c);
    k_reduce_final<true><<<1, RED_THREADS, 0, s>>>(c->red, 1, c->red_out), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("scaled_max");
    MB_CUDA(cudaMemcpyAsync(c->h_red, c->red_out, 8, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    *out = c->h_red[0];
    return MB_OK;
}

__global__ void __launch_bounds__(RED_THREADS)
k_functionals(Dims D, const uint32_t* __restrict__ vc, const double* __restrict__ u, double* partials) {
    // 0: sum Phi over last layer, 1: sum c over G, 2: sum c over E,G,K, 3: sum n, 4: count G
    double acc[5] = {0, 0, 0, 0, 0};
    int64_t n = D.N + D.F;
    int64_t last0 = (int64_t)(D.nt - 1) * D.syz;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < D.N) {
            int l = vc_phase(vc[i]);
            if (i >= last0) acc[0] += u[D.N + i];
            if (l == PG) { acc[1] += u[i]; acc[4] += 1.0; }
            if (has_c(l)) acc[2] += u[i];
        } else {
            acc[3] += u[2 * D.N + (i - D.N)];
        }
    }
    block_reduce_store<5, false>(acc, partials);
}

int functionals(mb_cell* c, const double* u, mb_step_info* info) {
    cudaStream_t s = c->stream;
    k_functionals<<<RED_BLOCKS, RED_THREADS, 0, s>>>(c->D, c->vcode, u, c->red), ::mb::count_launch(c);
    k_reduce_final<false><<<5, RED_THREADS, 0, s>>>(c->red, 5, c->red_out), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("functionals");
    MB_CUDA(cudaMemcpyAsync(c->h_red, c->red_out, 5 * 8, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    const double* h = c->h_red;
    double V = c->P.V, A = c->P.A;
    info->V_cell = h[0] / (double)c->D.syz;
    info->mean_c_solid = h[4] > 0 ? h[1] / h[4] : 0.0;
    info->Li_total = V * h[2] + A * h[3];
    info->Li_anode = V * h[1] + A * h[3];
    info->Li_plated = A * h[3];
    return MB_OK;
}

__global__ void __launch_bounds__(RED_THREADS)
k_count_diff(const uint8_t* __restrict__ a, const uint8_t* __restrict__ b, int64_t n, double* partials) {
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[0] += (a[i] != b[i]) ? 1.0 : 0.0;
    block_reduce_store<1, false>(acc, partials);
}

int count_diff_u8(mb_cell* c, const uint8_t* a, const uint8_t* b, int64_t n, int64_t* out) {
    if (n == 0) { *out = 0; return MB_OK; }
    cudaStream_t s = c->stream;
    k_count_diff<<<RED_BLOCKS, RED_THREADS, 0, s>>>(a, b, n, c->red), ::mb::count_launch(c);
    k_reduce_final<false><<<1, RED_THREADS, 0, s>>>(c->red, 1, c->red_out), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("count_diff");
    MB_CUDA(cudaMemcpyAsync(c->h_red, c->red_out, 8, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    *out = (int64_t)c->h_red[0];
    return MB_OK;
}

}  // namespace mb
