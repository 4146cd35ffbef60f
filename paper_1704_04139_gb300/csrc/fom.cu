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
// Pass 1: per voxel, mask of electrolyte neighbours of solid voxels with
// interface kinetics (G, K, L), the number of plating faces it owns (G) and
// the number of its other interface faces (K, L); flags forbidden contacts.
__global__ void k_classify_count(Dims D, const uint8_t* __restrict__ lab, uint8_t* __restrict__ emask,
                                 uint32_t* __restrict__ cnt, uint32_t* __restrict__ cnt2, int* __restrict__ err) {
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
        if ((lv == PG || lv == PK || lv == PL) && lw == PE) m |= 1u << d;
        // collector contacts with electrode solid (bit 2: CN, bit 3: CP)
        if (lv == PCN && (lw == PG || lw == PL)) atomicOr(err, 4);
        if (lv == PCP && (lw == PK || lw == PL)) atomicOr(err, 8);
    }
    emask[v] = (uint8_t)m;
    cnt[v] = lv == PG ? __popc(m) : 0u;
    cnt2[v] = lv == PG ? 0u : __popc(m);
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

// Pass 2: per-voxel code and the plating face list.  Interface faces are
// numbered plating faces first (G voxels, [0, F)), then the faces of K and L
// voxels ([F, NI)), each group by solid voxel index, then direction.
__global__ void k_classify_write(Dims D, const uint8_t* __restrict__ lab, const uint8_t* __restrict__ emask,
                                 const uint32_t* __restrict__ fbase, const uint32_t* __restrict__ kbase,
                                 uint32_t* __restrict__ vcode, int32_t* __restrict__ if_s,
                                 int32_t* __restrict__ if_e, int8_t* __restrict__ pf_dir) {
    int z, y, t;
    vox_coords(D, z, y, t);
    if (z >= D.nz || y >= D.ny) return;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    uint32_t m = emask[v];
    const bool g = lab[v] == PG;
    uint32_t fb = g ? fbase[v] : (m ? (uint32_t)D.F + kbase[v] : 0u);
    vcode[v] = (uint32_t)lab[v] | (m << 3) | (fb << VC_FBASE_SHIFT);
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    uint32_t f = fb;
    for (int d = 0; d < 6; ++d) {
        if (m & (1u << d)) {
            if_s[f] = (int32_t)v;
            if_e[f] = (int32_t)(v + off[d]);
            if (g) pf_dir[f] = (int8_t)d;
            ++f;
        }
    }
}

// Thread order of the stencil kernels whose per-face work depends on the
// phases of the face's two voxels (residual, Krylov operator): within each
// z-line (t, y) the voxels are ordered by (phase, whether a neighbour is of
// the other kind: electrolyte vs solid), stable in z.  A warp then mostly
// holds voxels of one phase and one contact type, so it executes one or two
// of the per-face branches per direction instead of all of them (a warp pays
// for every branch any of its lanes takes; the FP64 residual is bound by that
// on GB300's narrow FP64 pipe).  Every voxel's arithmetic is unchanged; the
// accesses stay within the line's few cache lines.  One thread per line.
__global__ void k_zperm(Dims D, const uint32_t* __restrict__ vc, uint16_t* __restrict__ zperm) {
    const int64_t line = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= (int64_t)D.nt * D.ny) return;
    const int t = (int)(line / D.ny), y = (int)(line % D.ny);
    const int64_t base = line * D.nz;   // = t * syz + y * nz
    constexpr int NKEY = 12;
    int cnt[NKEY];
#pragma unroll
    for (int k = 0; k < NKEY; ++k) cnt[k] = 0;
    auto key = [&](int z) {
        const int64_t v = base + z;
        const int lv = vc_phase(vc[v]);
        const bool el = lv == PE;
        bool mixed = false;
        if (t > 0) mixed |= (vc_phase(vc[v - D.syz]) == PE) != el;
        if (t < D.nt - 1) mixed |= (vc_phase(vc[v + D.syz]) == PE) != el;
        if (y > 0) mixed |= (vc_phase(vc[v - D.nz]) == PE) != el;
        if (y < D.ny - 1) mixed |= (vc_phase(vc[v + D.nz]) == PE) != el;
        if (z > 0) mixed |= (vc_phase(vc[v - 1]) == PE) != el;
        if (z < D.nz - 1) mixed |= (vc_phase(vc[v + 1]) == PE) != el;
        return 2 * lv + (mixed ? 1 : 0);
    };
    for (int z = 0; z < D.nz; ++z) {
        const int k = key(z);
#pragma unroll
        for (int q = 0; q < NKEY; ++q) cnt[q] += (q == k);
    }
    int start[NKEY];
    int acc = 0;
#pragma unroll
    for (int q = 0; q < NKEY; ++q) {
        start[q] = acc;
        acc += cnt[q];
    }
    for (int z = 0; z < D.nz; ++z) {
        const int k = key(z);
        int pos = 0;
#pragma unroll
        for (int q = 0; q < NKEY; ++q)
            if (q == k) pos = start[q]++;
        zperm[base + pos] = (uint16_t)z;
    }
}

int launch_classify(mb_cell* c, const uint8_t* d_lab) {
    const Dims& D = c->D;
    cudaStream_t s = c->stream;
    int64_t N = D.N;
    int64_t nb = (N + SCAN_B - 1) / SCAN_B;
    uint8_t* emask = nullptr;
    uint32_t *cnt = nullptr, *cnt2 = nullptr, *fbase = nullptr, *kbase = nullptr, *bsum = nullptr,
             *total = nullptr;
    int* err = nullptr;
    MB_CUDA(cudaMalloc(&emask, N));
    MB_CUDA(cudaMalloc(&cnt, N * 4));
    MB_CUDA(cudaMalloc(&cnt2, N * 4));
    MB_CUDA(cudaMalloc(&fbase, N * 4));
    MB_CUDA(cudaMalloc(&kbase, N * 4));
    MB_CUDA(cudaMalloc(&bsum, nb * 4 + 16));
    MB_CUDA(cudaMalloc(&total, 16));
    MB_CUDA(cudaMalloc(&err, 16));
    MB_CUDA(cudaMemsetAsync(err, 0, 4, s));
    k_classify_count<<<vox_grid(D, VOX_BLOCK), VOX_BLOCK, 0, s>>>(D, d_lab, emask, cnt, cnt2, err), ::mb::count_launch(c);
    k_scan_blocks<<<(unsigned)nb, SCAN_T, 0, s>>>(cnt, N, fbase, bsum), ::mb::count_launch(c);
    k_scan_sums<<<1, 1024, 0, s>>>(bsum, nb, total), ::mb::count_launch(c);
    k_scan_add<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(fbase, N, bsum), ::mb::count_launch(c);
    k_scan_blocks<<<(unsigned)nb, SCAN_T, 0, s>>>(cnt2, N, kbase, bsum), ::mb::count_launch(c);
    k_scan_sums<<<1, 1024, 0, s>>>(bsum, nb, total + 1), ::mb::count_launch(c);
    k_scan_add<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(kbase, N, bsum), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("classify");
    int h_err = 0;
    uint32_t h_tot[2] = {0, 0};
    MB_CUDA(cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaMemcpyAsync(h_tot, total, 8, cudaMemcpyDeviceToHost, s));
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
    } else if ((uint64_t)h_tot[0] + h_tot[1] >= VC_MAX_FACES) {
        set_error("too many interface faces for the 23-bit face index");
        rc = MB_EINVAL;
    }
    const uint32_t h_total = h_tot[0];
    if (rc == MB_OK) {
        c->D.F = h_total;
        c->D.NI = (int64_t)h_tot[0] + h_tot[1];
        c->n = 2 * N + (int64_t)h_total;
        size_t F = h_total ? h_total : 1;
        size_t NI = c->D.NI ? (size_t)c->D.NI : 1;
        c->vcode = (uint32_t*)cell_alloc(c, N * 4);
        c->zperm = (uint16_t*)cell_alloc(c, N * 2);
        // interface face list; the plating faces are its first F entries
        c->if_s = (int32_t*)cell_alloc(c, NI * 4);
        c->if_e = (int32_t*)cell_alloc(c, NI * 4);
        c->pf_g = c->if_s;
        c->pf_e = c->if_e;
        c->pf_dir = (int8_t*)cell_alloc(c, F);
        if (!c->vcode || !c->zperm || !c->if_s || !c->if_e || !c->pf_dir) rc = MB_ENOMEM;
    }
    if (rc == MB_OK) {
        k_classify_write<<<vox_grid(D, VOX_BLOCK), VOX_BLOCK, 0, s>>>(
            c->D, d_lab, emask, fbase, kbase, c->vcode, c->if_s, c->if_e, c->pf_dir), ::mb::count_launch(c);
        const int64_t lines = (int64_t)D.nt * D.ny;
        k_zperm<<<(unsigned)((lines + 127) / 128), 128, 0, s>>>(c->D, c->vcode, c->zperm), ::mb::count_launch(c);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "classify_write");
    }
    cudaStreamSynchronize(s);
    cudaFree(emask); cudaFree(cnt); cudaFree(cnt2); cudaFree(fbase); cudaFree(kbase); cudaFree(bsum);
    cudaFree(total); cudaFree(err);
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
k_residual(ParT<T> P, Dims D, const uint32_t* __restrict__ vc, const T* __restrict__ u,
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

// Residual in two passes (the solver's Newton residual): k_iface_current
// evaluates the Butler-Volmer and plating current densities of every
// interface face once (FP64; the transcendental part of the residual), then
// k_residual_split assembles every voxel's rows from them and the bulk and
// conduction fluxes.  Same arithmetic per term as k_residual (which
// evaluates each interface current twice, once from each side; the C-ABI
// residual entry points use that single-kernel form) except the migration
// flux's 1/(c_v + c_w), taken by rcp_nr (~1 ulp) instead of a division.
__global__ void __launch_bounds__(256)
k_iface_current(DevParams P, Dims D, const uint32_t* __restrict__ vc, const int32_t* __restrict__ if_s,
                const int32_t* __restrict__ if_e, const double* __restrict__ u, const uint8_t* __restrict__ gate,
                double s_i0, double k_pl, double* __restrict__ icur) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = D.N, NI = D.NI;
    if (i >= NI) return;
    const int64_t v = if_s[i], w = if_e[i];
    double nf = 0.0;
    bool g = false;
    if (i < D.F) {   // plating face
        nf = u[2 * N + i];
        g = gate[i] != 0;
    }
    double ibv, ipl;
    interface_current<double>(P, vc_phase(vc[v]), u[v], u[N + v], u[w], u[N + w], nf, g, s_i0, k_pl, ibv, ipl);
    icur[i] = ibv;
    icur[NI + i] = ipl;
}

__global__ void __launch_bounds__(256)
k_residual_split(DevParams P, Dims D, const uint32_t* __restrict__ vc, const uint16_t* __restrict__ zperm,
                 const double* __restrict__ u, const double* __restrict__ uold, const double* __restrict__ icur,
                 double dt_inv, double I_app, double* __restrict__ r) {
    // the phase-indexed coefficient tables in shared memory: indexed by the
    // threads' own phases, kernel-parameter (constant bank) loads would be
    // serialised over the distinct phases of a warp
    __shared__ double s_gD[6], s_gs[36];
    {
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        if (tid < 6) s_gD[tid] = P.gD[tid];
        if (tid < 36) s_gs[tid] = P.gsig[tid / 6][tid % 6];
        __syncthreads();
    }
    int z, y, t;
    vox_coords(D, z, y, t);
    if (z >= D.nz || y >= D.ny) return;
    z = zperm[((int64_t)t * D.ny + y) * D.nz + z];   // grouped thread order (k_zperm)
    const int64_t N = D.N, NI = D.NI;
    int64_t v = (int64_t)t * D.syz + (int64_t)y * D.nz + z;
    const uint32_t code = vc[v];
    const int lv = vc_phase(code);
    const double cv = u[v], pv = u[N + v];
    double rc = 0.0, rp = 0.0;
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
    int64_t ibase = vc_fbase(code);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (!inb[d]) continue;
        const int64_t w = v + off[d];
        const uint32_t cw_code = vc[w];
        const int lw = vc_phase(cw_code);
        if (lv == PE && lw == PE) {
            const double cw = u[w], pw = u[N + w];
            const double S = fmax(cv, P.cmin[PE]) + fmax(cw, P.cmin[PE]);
            const double dc = cw - cv, dp = pw - pv;
            const double j = -P.E_gk * dp - P.E_gm * dc * rcp_nr(S);
            rc += -P.E_gD * dc + P.E_tF * j;
            rp += j;
        } else if (lv == lw && (lv == PG || lv == PK)) {
            rc += -s_gD[lv] * (u[w] - cv);
            rp += -s_gs[lv * 6 + lw] * (u[N + w] - pv);
        } else if (lv != PE && lw != PE) {
            rp += -s_gs[lv * 6 + lw] * (u[N + w] - pv);
        } else if (lw == PE && (lv == PG || lv == PK || lv == PL)) {
            const int64_t i = ibase++;
            const double ibv = icur[i], ipl = icur[NI + i];
            if (lv != PL) rc += P.A * ibv * P.invF;
            rp += P.A * (ibv + ipl);
            if (lv == PG) r[2 * N + i] = (u[2 * N + i] - uold[2 * N + i]) * dt_inv + ipl * P.invF;
        } else if (lv == PE && (lw == PG || lw == PK || lw == PL)) {
            const int64_t i = (int64_t)vc_fbase(cw_code) + __popc(vc_emask(cw_code) & ((1u << opp_dir(d)) - 1u));
            const double it = icur[i] + icur[NI + i];
            rc -= P.A * it * P.invF;
            rp -= P.A * it;
        }
    }
    if (t == 0 && lv == PCN) rp += P.g_dir * pv;
    if (t == D.nt - 1 && lv == PCP) rp += P.A * I_app;
    if (has_c(lv)) rc += P.V * (cv - uold[v]) * dt_inv;
    else rc = cv;
    r[v] = rc;
    r[N + v] = rp;
}

int launch_residual_split(mb_cell* c, const double* u, const double* u_old, const uint8_t* gate, double dt,
                          double I_app, double* r, cudaStream_t s) {
    const Dims& D = c->D;
    cudaEvent_t ev;
    prof_begin(c, s, &ev);
    if (D.NI)
        k_iface_current<<<(unsigned)((D.NI + 255) / 256), 256, 0, s>>>(c->P, D, c->vcode, c->if_s, c->if_e, u, gate,
                                                                       c->s_i0, c->k_pl, c->icur), ::mb::count_launch(c);
    k_residual_split<<<vox_grid(D, VOX_BLOCK), VOX_BLOCK, 0, s>>>(c->P, D, c->vcode, c->zperm, u, u_old, c->icur,
                                                                  1.0 / dt, I_app, r), ::mb::count_launch(c);
    prof_end(c, s, PROF_RESIDUAL, ev);
    MB_CUDA_LAUNCH("residual_split");
    return MB_OK;
}

template <class T>
int launch_residual(mb_cell* c, const T* u, const double* u_old, const uint8_t* gate, double dt,
                    double I_app, T* r, cudaStream_t s) {
    const Dims& D = c->D;
    cudaEvent_t ev;
    prof_begin(c, s, &ev);
    k_residual<T><<<vox_grid(D, VOX_BLOCK), VOX_BLOCK, 0, s>>>(cell_par<T>(c), D, c->vcode, u, u_old, gate,
                                                               1.0 / dt, I_app, c->s_i0, c->k_pl, r), ::mb::count_launch(c);
    prof_end(c, s, PROF_RESIDUAL, ev);
    MB_CUDA_LAUNCH("residual");
    return MB_OK;
}
template int launch_residual<double>(mb_cell*, const double*, const double*, const uint8_t*, double,
                                     double, double*, cudaStream_t);

// ------------------------------------------------------------ K2: JVP
// J(u) v from the analytic per-face partial derivatives (chain rule through
// sqrt, sinh, cosh, exp, 1/cbar, U0'(c) and f_pre'(n)).
// With SCALED, x is in scaled unknowns (x_hat = x / s_u) and each output row
// is divided by the residual scale s_r and by the magnitude of its own
// diagonal entry in these units: the Krylov operator E S_r^-1 J S_u with
// E = |diag(S_r^-1 J S_u)|^-1, so that every row of the Krylov system has a
// unit diagonal whatever its physical scale (collector and electrolyte rows
// differ by ~1e10 otherwise).
// k_jvp: direction and result in one precision TV (the FP64 and FP32 JVPs of
// the C-ABI), all per-face coefficients evaluated on the fly.  TC: precision
// of the linearisation point and of the nonlinear per-face coefficients.  The
// solver itself uses the stencil form k_jvp_lin below.
template <class TC, class TV, int MODE>
__global__ void __launch_bounds__(256)
k_jvp(ParT<TC> P, Dims D, const uint32_t* __restrict__ vc, const TC* __restrict__ u,
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
    const TV nc = TV(P.nc);
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
        face_jvp<TC, TV>(P, lv, lw, cv, pv, cw, pw, nf, g, s_i0, k_pl, dcv, dcw, dcw - dcv, dpw - dpv, dnf, jc, jp,
                         jn, jnn, dgc, dgp);
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
    const TV Vdt = TV(P.V) * idt;
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
    const ParT<TC>& P = cell_par<TC>(c);
    cudaEvent_t ev;
    prof_begin(c, s, &ev);
    if (mode == 2)
        k_jvp<TC, TV, 2><<<g, VOX_BLOCK, 0, s>>>(P, D, c->vcode, u, gate, 1.0 / dt, c->s_i0, c->k_pl, v, jv), ::mb::count_launch(c);
    else if (mode == 1)
        k_jvp<TC, TV, 1><<<g, VOX_BLOCK, 0, s>>>(P, D, c->vcode, u, gate, 1.0 / dt, c->s_i0, c->k_pl, v, jv), ::mb::count_launch(c);
    else
        k_jvp<TC, TV, 0><<<g, VOX_BLOCK, 0, s>>>(P, D, c->vcode, u, gate, 1.0 / dt, c->s_i0, c->k_pl, v, jv), ::mb::count_launch(c);
    prof_end(c, s, PROF_JVP, ev);
    MB_CUDA_LAUNCH("jvp");
    return MB_OK;
}
template int launch_jvp<double, double>(mb_cell*, const double*, const uint8_t*, double, const double*, double*,
                                        cudaStream_t, int);
template int launch_jvp<float, float>(mb_cell*, const float*, const uint8_t*, double, const float*, float*,
                                      cudaStream_t, int);

// ------------------------------------------- K2': linearised JVP (stencil)
// The interface kinetics are the only costly part of the Jacobian (sqrt,
// sinh, cosh, exp, the OCP and its derivative) and they are fixed during a
// linear solve: k_lin_setup evaluates their six partial derivatives once per
// interface face, and k_jvp_lin applies the Jacobian as a stencil on them.
// One thread per voxel; solid voxels with electrolyte neighbours write the
// partials of their own interface faces.
// One thread per interface face (solid voxel if_s[i], electrolyte voxel
// if_e[i]); faces [0, F) are the plating faces.
template <class TC>
__global__ void __launch_bounds__(256)
k_lin_setup(ParT<TC> P, Dims D, const uint32_t* __restrict__ vc, const int32_t* __restrict__ if_s,
            const int32_t* __restrict__ if_e, const TC* __restrict__ u, const uint8_t* __restrict__ gate,
            double s_i0d, double k_pld, float* __restrict__ icoef) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = D.N, NI = D.NI;
    if (i >= NI) return;
    const int64_t v = if_s[i], w = if_e[i];
    const int lv = vc_phase(vc[v]);
    const TC s_i0 = TC(s_i0d), k_pl = TC(k_pld);
    TC nf = TC(0);
    bool g = false;
    if (i < D.F) {   // plating face
        nf = u[2 * N + i];
        g = gate[i] != 0;
    }
    TC i_eta, i_cs, i_ce, ip_eta, ip_ce, ip_n;
    interface_partials<TC>(P, lv, u[v], u[N + v], u[w], u[N + w], nf, g, s_i0, k_pl, i_eta, i_cs, i_ce, ip_eta,
                           ip_ce, ip_n);
    icoef[0 * NI + i] = float(i_eta);
    icoef[1 * NI + i] = float(ip_eta);
    icoef[2 * NI + i] = float(i_cs);
    icoef[3 * NI + i] = float(i_ce);
    icoef[4 * NI + i] = float(ip_ce);
    icoef[5 * NI + i] = float(ip_n);
}

template <class TC>
int launch_lin_setup(mb_cell* c, const TC* u, const uint8_t* gate, cudaStream_t s) {
    const Dims& D = c->D;
    if (D.NI == 0) return MB_OK;
    k_lin_setup<TC><<<(unsigned)((D.NI + 255) / 256), 256, 0, s>>>(cell_par<TC>(c), D, c->vcode, c->if_s, c->if_e, u,
                                                                   gate, c->s_i0, c->k_pl, c->icoef), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("lin_setup");
    return MB_OK;
}
template int launch_lin_setup<float>(mb_cell*, const float*, const uint8_t*, cudaStream_t);
template int launch_lin_setup<double>(mb_cell*, const double*, const uint8_t*, cudaStream_t);

// J v on a float-float direction in scaled units: output rows divided by the
// residual scale s_r and by the row equilibration (multiplied by rowinv): the
// Krylov operator, face rows written.  FP32 arithmetic; differences taken before
// rounding (see face_jvp).  Each face first selects its coefficients on
// (dphi_w - dphi_v, dc_w - dc_v, dc_v, dc_w, dn_f) for the phi and c rows in a
// short branch, then all faces share one update, so that a warp of mixed
// phases pays little for divergence.  scal: [0] 1/dt, [1 + phase]
// 1/(V c_ref/dt), [7] 1/A, [8] dt/n_c.
__global__ void __launch_bounds__(256, 4)
k_jvp_lin(ParT<float> P, Dims D, const uint32_t* __restrict__ vc, const uint16_t* __restrict__ zperm,
          const float* __restrict__ c32,
          const float* __restrict__ icoef, const float* __restrict__ rowinv, const float* __restrict__ scal,
          const float2* __restrict__ x, float* __restrict__ y_out) {
    // phase-indexed tables and the solve's scalars in shared memory (indexed
    // by the threads' own phases; see k_residual_split)
    __shared__ float s_cref[6], s_gD[6], s_gs[36], s_scal[9];
    {
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        if (tid < 6) {
            s_cref[tid] = P.cref[tid];
            s_gD[tid] = P.gD[tid];
        }
        if (tid < 36) s_gs[tid] = P.gsig[tid / 6][tid % 6];
        if (tid < 9) s_scal[tid] = scal[tid];
        __syncthreads();
    }
    int z, y, t;
    vox_coords(D, z, y, t);
    if (z >= D.nz || y >= D.ny) return;
    z = zperm[((int64_t)t * D.ny + y) * D.nz + z];   // grouped thread order (k_zperm)
    const int syz = (int)D.syz, nz = D.nz;
    const int NI = (int)D.NI;
    const int v = t * syz + y * nz + z;
    const float2* __restrict__ xp = x + D.N;        // potentials
    const float2* __restrict__ xn = x + 2 * D.N;    // plating faces
    const float dt_inv = s_scal[0];
    const uint32_t code = vc[v];
    const int lv = vc_phase(code);
    const float crv = s_cref[lv], crE = P.cref[PE];
    const float2 xcv = x[v], xpv = xp[v];
    const float dcv = df_val(xcv) * crv, dpv = df_val(xpv);
    const float A = P.A, AF = P.A * P.invF;
    const bool vkin = lv == PG || lv == PK || lv == PL;
    float jc = 0.f, jp = 0.f;
    const int off[6] = {-syz, syz, -nz, nz, -1, 1};
    const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
    int ibase = (int)vc_fbase(code);
    // all neighbour loads first (indices clamped to v outside the grid), so
    // that they are in flight together
    uint32_t cwc[6];
    float2 xpn[6], xcn[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const int w = inb[d] ? v + off[d] : v;
        cwc[d] = vc[w];
        xpn[d] = xp[w];
        xcn[d] = x[w];
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        if (!inb[d]) continue;
        const int w = v + off[d];
        const uint32_t cw_code = cwc[d];
        const int lw = vc_phase(cw_code);
        const float ddp = df_diff(xpn[d], xpv);
        const float2 xcw = xcn[d];
        float p1 = 0.f, p2 = 0.f, p3 = 0.f, p4 = 0.f, p5 = 0.f;   // phi row
        float q1 = 0.f, q2 = 0.f, q3 = 0.f, q4 = 0.f, q5 = 0.f;   // c row
        float ddc = 0.f, dcw = 0.f, dnf = 0.f;
        if (lv == PE && lw == PE) {
            ddc = df_diff(xcw, xcv) * crE;
            dcw = df_val(xcw) * crE;
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
            ddc = df_diff(xcw, xcv) * crv;
            q2 = -s_gD[lv];
            p1 = -s_gs[lv * 6 + lw];
        } else if (lv != PE && lw != PE) {
            p1 = -s_gs[lv * 6 + lw];   // conduction between electronic conductors
        } else if (vkin && lw == PE) {
            // solid v next to electrolyte w: interface face ibase (deta = -ddp)
            const int i = ibase++;
            const float i_eta = icoef[i], ip_eta = icoef[NI + i], i_cs = icoef[2 * NI + i];
            const float i_ce = icoef[3 * NI + i], ip_ce = icoef[4 * NI + i], ip_n = icoef[5 * NI + i];
            dcw = df_val(xcw) * crE;
            if (lv == PG) dnf = df_val(xn[i]) * P.nc;
            p1 = -A * (i_eta + ip_eta);
            p3 = A * i_cs;
            p4 = A * (i_ce + ip_ce);
            p5 = A * ip_n;
            if (lv != PL) {
                q1 = -AF * i_eta;
                q3 = AF * i_cs;
                q4 = AF * i_ce;
            }
            if (lv == PG) {
                const float dipl = -ip_eta * ddp + ip_ce * dcw + ip_n * dnf;
                y_out[2 * D.N + i] = (P.invF * dipl + dnf * dt_inv) * s_scal[8] * rowinv[2 * D.N + i];
            }
        } else if (lv == PE && (lw == PG || lw == PK || lw == PL)) {
            // electrolyte v next to solid w: di = (i_eta + ip_eta) ddp + i_cs dc_w + (i_ce + ip_ce) dc_v + ip_n dn
            const int i = (int)vc_fbase(cw_code) + __popc(vc_emask(cw_code) & ((1u << opp_dir(d)) - 1u));
            const float i_eta = icoef[i], ip_eta = icoef[NI + i], i_cs = icoef[2 * NI + i];
            const float i_ce = icoef[3 * NI + i], ip_ce = icoef[4 * NI + i], ip_n = icoef[5 * NI + i];
            dcw = df_val(xcw) * s_cref[lw];
            if (lw == PG) dnf = df_val(xn[i]) * P.nc;
            p1 = -A * (i_eta + ip_eta);
            p3 = -A * (i_ce + ip_ce);
            p4 = -A * i_cs;
            p5 = -A * ip_n;
            q1 = -AF * (i_eta + ip_eta);
            q3 = -AF * (i_ce + ip_ce);
            q4 = -AF * i_cs;
            q5 = -AF * ip_n;
        }
        jp += p1 * ddp + p2 * ddc + p3 * dcv + p4 * dcw + p5 * dnf;
        jc += q1 * ddp + q2 * ddc + q3 * dcv + q4 * dcw + q5 * dnf;
    }
    if (t == 0 && lv == PCN) jp += P.g_dir * dpv;
    if (has_c(lv)) jc = (jc + P.V * dt_inv * dcv) * s_scal[1 + lv];
    else jc = dcv;
    jp *= s_scal[7];
    jc *= rowinv[v];
    jp *= rowinv[D.N + v];
    y_out[v] = jc;
    y_out[D.N + v] = jp;
}

// per-solve scalars of k_jvp_lin (layout there), one thread
__global__ void k_set_scal(DevParams P, double dt, float* scal) {
    const double idt = 1.0 / dt;
    scal[0] = float(idt);
    for (int l = 0; l < 6; ++l) scal[1 + l] = float(1.0 / (P.V * idt * P.cref[l]));
    scal[7] = float(1.0 / P.A);
    scal[8] = float(1.0 / (P.nc * idt));
}

int set_dt(mb_cell* c, double dt, cudaStream_t s) {
    k_set_scal<<<1, 1, 0, s>>>(c->P, dt, c->d_dtinv), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("set_dt");
    return MB_OK;
}

int launch_jvp_lin(mb_cell* c, const float2* v, float* jv, cudaStream_t s) {
    const Dims& D = c->D;
    const dim3 g = vox_grid(D, VOX_BLOCK);
    const float* sc = c->d_dtinv;
    cudaEvent_t ev;
    prof_begin(c, s, &ev);
    k_jvp_lin<<<g, VOX_BLOCK, 0, s>>>(c->Pf, D, c->vcode, c->zperm, c->u32, c->icoef, c->rowinv, sc, v, jv),
        ::mb::count_launch(c);
    prof_end(c, s, PROF_JVP, ev);
    MB_CUDA_LAUNCH("jvp_lin");
    return MB_OK;
}

// ------------------------------------------------------------ plating gates
// g_f = 1 where plated Li is present (n_old > 1e-9 n_c: smaller inventories
// count as none, f_pre ~ 1e-36 there) or the plating overpotential
// Phi_G - phi_E is negative (Sec. workflow:degradation_modeling).
__global__ void k_gate(Dims D, const int32_t* __restrict__ pg, const int32_t* __restrict__ pe,
                       const double* __restrict__ u, const double* __restrict__ n_old, double n_gate,
                       uint8_t* __restrict__ gate) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= D.F) return;
    const double* ph = u + D.N;
    double etap = ph[pg[f]] - ph[pe[f]];
    gate[f] = (n_old[f] > n_gate || etap < 0.0) ? 1 : 0;
}

int launch_gate(mb_cell* c, const double* u, const double* n_old, uint8_t* gate, cudaStream_t s) {
    if (c->D.F == 0) return MB_OK;
    k_gate<<<(unsigned)((c->D.F + 255) / 256), 256, 0, s>>>(c->D, c->pf_g, c->pf_e, u, n_old, GATE_N_REL * c->P.nc, gate), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("gate");
    return MB_OK;
}

int launch_gate_residual_unprofiled(mb_cell* c, const double* u, const double* u_old, uint8_t* gate_scratch,
                                    double dt, double I_app, double* r, cudaStream_t s) {
    const Dims& D = c->D;
    if (D.F > 0) {
        k_gate<<<(unsigned)((D.F + 255) / 256), 256, 0, s>>>(D, c->pf_g, c->pf_e, u_old, u_old + 2 * D.N,
                                                             GATE_N_REL * c->P.nc, gate_scratch), ::mb::count_launch(c);
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
k_scaled_max(Dims D, const uint32_t* __restrict__ vc, const double* __restrict__ x, InvScales is, double nc,
             const double* __restrict__ u, double* partials) {
    // [0] over every unknown; [1] the step-length cap: the voxel unknowns (c, phi)
    // in their scales and, with u given, each plated inventory relative to
    // max(n_c, |n_f|) of the state u.
    // The scale is constant per class (concentration by phase, potential,
    // inventory), so the loop keeps the largest |x| per class as an integer
    // maximum of the FP64 bit patterns with the sign cleared (for non-negative
    // doubles the integer order is the numeric order, and NaN patterns sort
    // above infinity), and scales once at the end: no FP64 arithmetic per
    // element.  The relative cap term is formed in FP32 (a step-length
    // heuristic; FP32 resolves it far beyond its 0.25 threshold).
    constexpr unsigned long long ABS = 0x7fffffffffffffffull;
    unsigned long long mc[6] = {0, 0, 0, 0, 0, 0}, mp = 0, mn = 0;
    float capn = 0.f;
    const float ncf = (float)nc;
    int64_t n = 2 * D.N + D.F;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(x[i]) & ABS;
        if (i < D.N) {
            const int ph = vc_phase(vc[i]);
#pragma unroll
            for (int k = 0; k < 6; ++k)
                if (ph == k) mc[k] = b > mc[k] ? b : mc[k];
        } else if (i < 2 * D.N) {
            mp = b > mp ? b : mp;
        } else {
            mn = b > mn ? b : mn;
            if (u) {
                const float ac = (float)__longlong_as_double((long long)b) / fmaxf(ncf, fabsf((float)u[i]));
                capn = (ac == ac) ? fmaxf(capn, ac) : INFINITY;
            }
        }
    }
    auto scaled = [](unsigned long long m, double sc) {
        const double a = __longlong_as_double((long long)m) * sc;
        return (a == a) ? a : 1e300;   // NaN -> huge
    };
    double vox = scaled(mp, is.phi);
#pragma unroll
    for (int k = 0; k < 6; ++k) vox = fmax(vox, scaled(mc[k], is.c[k]));
    double acc[2];
    acc[0] = fmax(vox, scaled(mn, is.n));
    acc[1] = u ? fmax(vox, capn < INFINITY ? (double)capn : 1e300) : vox;
    block_reduce_store<2, true>(acc, partials);
}

InvScales inv_scales(const mb_cell* c, int which, double dt) {
    InvScales is;
    const DevParams& P = c->P;
    for (int l = 0; l < 6; ++l)
        is.c[l] = which == 0 ? 1.0 / P.cref[l] : (has_c(l) ? dt / (P.V * P.cref[l]) : 1.0);
    is.phi = which == 0 ? 1.0 : 1.0 / P.A;
    is.n = which == 0 ? 1.0 / P.nc : dt / P.nc;
    return is;
}

int scaled_maxnorm(mb_cell* c, const double* x, int which, double dt, double* out, double* out_cap,
                   const double* u_cap) {
    cudaStream_t s = c->stream;
    k_scaled_max<<<RED_BLOCKS, RED_THREADS, 0, s>>>(c->D, c->vcode, x, inv_scales(c, which, dt), c->P.nc, u_cap,
                                                    c->red), ::mb::count_launch(c);
    k_reduce_final<true><<<2, RED_THREADS, 0, s>>>(c->red, 2, c->red_out), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("scaled_max");
    MB_CUDA(cudaMemcpyAsync(c->h_red, c->red_out, 16, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    *out = c->h_red[0];
    if (out_cap) *out_cap = c->h_red[1];
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
