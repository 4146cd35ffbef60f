// rom_build.cu -- offline construction of the reduced model (Sec.
// workflow:MOR) from full-order solves of the cell on the GPU.
//
// 1. Snapshots: full-order trajectories (mb_step) at the given parameter
//    points from the cell's current state, recording every Newton stage with
//    its plating gates (the paper includes the intermediate Newton stages).
// 2. POD of c, of the plated-Li inventory n and of phi separately in the
//    L^2 inner product of the grid (weight V per voxel value, A per face
//    value): Gram matrix of each block on the GPU, its eigen-decomposition on
//    the host (cyclic Jacobi), modes S X Lambda^-1/2 on the GPU, then two
//    Cholesky orthonormalisation passes in the weighted inner product.
// 3. Empirical interpolation (EI-Greedy): training columns are the interface
//    terms (Butler-Volmer of graphite and cathode at unit exchange-current
//    scale, the Li-foil counter electrode, and plating at unit rate with the
//    snapshot's gates) of every snapshot, in one common basis, and the
//    migration term with 1/c (Eq. phiel) of every snapshot; each step takes
//    the column with the largest max-norm interpolation error (ties: lowest
//    index), its largest entry as the point and the error column scaled to one
//    there as the basis vector.
// 4. Projections of Eq. ap4:fully_reduced with residual rows weighted by
//    (1, 1, A) for (c, phi, n) rows: storage, the linear part, the boundary
//    term, the interpolation bases Q (Q[P,:])^-1, and the output functionals.
// The result goes to mb_rom_create.  FP64 throughout; the Gram route limits
// the POD to singular values above ~1e-7 of the largest of each block.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mb_internal.h"

namespace mb {

// ---------------------------------------------------------------- kernels
__device__ inline void vox_ijk(const Dims& D, int64_t v, int& t, int& y, int& z) {
    z = (int)(v % D.nz);
    y = (int)((v / D.nz) % D.ny);
    t = (int)(v / D.syz);
}

// Nonlinear sub-operators of the residual at state u with plating gates g,
// each in the residual layout: out[0] Butler-Volmer of G and K (s_i0 = 1),
// out[1] Li-foil counter electrode, out[2] plating (k_pl = 1, gated),
// out[3] electrolyte migration with 1/cbar.  One thread per voxel; the face
// rows of plating are written by the graphite voxel.
__global__ void k_subops(DevParams P, Dims D, const uint32_t* __restrict__ vc, const double* __restrict__ u,
                         const uint8_t* __restrict__ gate, double* __restrict__ obv, double* __restrict__ oce,
                         double* __restrict__ opl, double* __restrict__ o1c) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= D.N) return;
    const int64_t N = D.N;
    int t, y, z;
    vox_ijk(D, v, t, y, z);
    const uint32_t code = vc[v];
    const int lv = vc_phase(code);
    const double cv = u[v], pv = u[N + v];
    double bc = 0, bp = 0, cc = 0, cp = 0, pc = 0, pp = 0, mc = 0, mp = 0;
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    const bool inb[6] = {t > 0, t < D.nt - 1, y > 0, y < D.ny - 1, z > 0, z < D.nz - 1};
    int64_t ibase = vc_fbase(code);
    const double A = P.A, invF = P.invF;
    for (int d = 0; d < 6; ++d) {
        if (!inb[d]) continue;
        const int64_t w = v + off[d];
        const uint32_t cw_code = vc[w];
        const int lw = vc_phase(cw_code);
        const double cw = u[w], pw = u[N + w];
        if (lv == PE && lw == PE) {
            const double S = fmax(cv, P.cmin[PE]) + fmax(cw, P.cmin[PE]);
            const double jm = -P.E_gm * (cw - cv) / S;          // A j_m, outflow from v
            mc += P.E_tF * jm;
            mp += jm;
        } else if (lw == PE && (lv == PG || lv == PK || lv == PL)) {
            const int64_t f = ibase++;
            double nf = 0.0;
            bool g = false;
            if (lv == PG) { nf = u[2 * N + f]; g = gate[f] != 0; }
            double ibv, ipl;
            interface_current<double>(P, lv, cv, pv, cw, pw, nf, g, 1.0, 1.0, ibv, ipl);
            if (lv == PL) {
                cp += A * ibv;
            } else {
                bc += A * ibv * invF;
                bp += A * ibv;
            }
            if (lv == PG) {
                pp += A * ipl;
                opl[2 * N + f] = ipl * invF;
            }
        } else if (lv == PE && (lw == PG || lw == PK || lw == PL)) {
            const int64_t f = (int64_t)vc_fbase(cw_code) + __popc(vc_emask(cw_code) & ((1u << opp_dir(d)) - 1u));
            double nf = 0.0;
            bool g = false;
            if (lw == PG) { nf = u[2 * N + f]; g = gate[f] != 0; }
            double ibv, ipl;
            interface_current<double>(P, lw, cw, pw, cv, pv, nf, g, 1.0, 1.0, ibv, ipl);
            if (lw == PL) {
                cc -= A * ibv * invF;
                cp -= A * ibv;
            } else {
                bc -= A * ibv * invF;
                bp -= A * ibv;
            }
            if (lw == PG) {
                pc -= A * ipl * invF;
                pp -= A * ipl;
            }
        }
    }
    obv[v] = bc; obv[N + v] = bp;
    oce[v] = cc; oce[N + v] = cp;
    opl[v] = pc; opl[N + v] = pp;
    o1c[v] = mc; o1c[N + v] = mp;
}

// y = A_lin x: diffusion, conduction, the potential part of the electrolyte
// flux, the collector ghost term and the identity rows of voxels without c
// (face rows zero).  One thread per voxel.
__global__ void k_lin_apply(DevParams P, Dims D, const uint32_t* __restrict__ vc, const double* __restrict__ x,
                            double* __restrict__ y) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= D.N) return;
    const int64_t N = D.N;
    int t, yy, z;
    vox_ijk(D, v, t, yy, z);
    const int lv = vc_phase(vc[v]);
    const double cv = x[v], pv = x[N + v];
    double rc = 0.0, rp = 0.0;
    const int64_t off[6] = {-D.syz, D.syz, -(int64_t)D.nz, (int64_t)D.nz, -1, 1};
    const bool inb[6] = {t > 0, t < D.nt - 1, yy > 0, yy < D.ny - 1, z > 0, z < D.nz - 1};
    for (int d = 0; d < 6; ++d) {
        if (!inb[d]) continue;
        const int64_t w = v + off[d];
        const int lw = vc_phase(vc[w]);
        const double dc = x[w] - cv, dp = x[N + w] - pv;
        if (lv == PE && lw == PE) {
            const double j = -P.E_gk * dp;
            rc += -P.E_gD * dc + P.E_tF * j;
            rp += j;
        } else if (lv == lw && (lv == PG || lv == PK)) {
            rc += -P.gD[lv] * dc;
            rp += -P.gsig[lv][lw] * dp;
        } else if (lv != PE && lw != PE) {
            rp += -P.gsig[lv][lw] * dp;
        }
    }
    if (t == 0 && lv == PCN) rp += P.g_dir * pv;
    if (!has_c(lv)) rc = cv;
    y[v] = rc;
    y[N + v] = rp;
}

// C (p x q, row-major) = A^T diag(w) B with A (L x p) and B (L x q) column-major
constexpr int GT = 16;
__global__ void k_atwb(int64_t L, int p, int q, const double* __restrict__ A, const double* __restrict__ B,
                       const double* __restrict__ w, double* __restrict__ C) {
    __shared__ double sa[GT][GT + 1], sb[GT][GT + 1];
    const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
    const int ty = threadIdx.y, tx = threadIdx.x;
    double acc = 0.0;
    for (int64_t l0 = 0; l0 < L; l0 += GT) {
        const int64_t l = l0 + tx;
        const int i = i0 + ty, j = j0 + ty;
        const double wl = (l < L) ? (w ? w[l] : 1.0) : 0.0;
        sa[ty][tx] = (i < p && l < L) ? A[(int64_t)i * L + l] * wl : 0.0;
        sb[ty][tx] = (j < q && l < L) ? B[(int64_t)j * L + l] : 0.0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GT; ++k) acc += sa[ty][k] * sb[tx][k];
        __syncthreads();
    }
    const int i = i0 + ty, j = j0 + tx;
    if (i < p && j < q) C[(int64_t)i * q + j] = acc;
}

// Y (L x r, column-major) = S (L x K, column-major) X (K x r, row-major)
__global__ void k_sx(int64_t L, int K, int r, const double* __restrict__ S, const double* __restrict__ X,
                     double* __restrict__ Y) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (l >= L) return;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc += S[(int64_t)k * L + l] * X[(int64_t)k * r + j];
    Y[(int64_t)j * L + l] = acc;
}

// per column j of R (L x K, column-major): max |R[:, j]|
__global__ void k_colmax(int64_t L, const double* __restrict__ R, double* __restrict__ out) {
    __shared__ double sh[256];
    const int j = blockIdx.x;
    double m = 0.0;
    for (int64_t l = threadIdx.x; l < L; l += blockDim.x) m = fmax(m, fabs(R[(int64_t)j * L + l]));
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = sh[0];
}

// index of the largest |col[l]| (lowest index on ties), one block
__global__ void k_argmax(int64_t L, const double* __restrict__ col, int64_t* __restrict__ out) {
    __shared__ double sv[256];
    __shared__ int64_t si[256];
    double best = -1.0;
    int64_t bi = 0;
    for (int64_t l = threadIdx.x; l < L; l += blockDim.x) {
        double a = fabs(col[l]);
        if (a > best) { best = a; bi = l; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double v2 = sv[threadIdx.x + s];
            int64_t i2 = si[threadIdx.x + s];
            if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = si[0];
}

// q = R[:, k] / R[p, k]
__global__ void k_ei_newvec(int64_t L, const double* __restrict__ R, int k, int64_t p, double* __restrict__ q) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l < L) q[l] = R[(int64_t)k * L + l] / R[(int64_t)k * L + p];
}

__global__ void k_getrow(int64_t L, int K, const double* __restrict__ R, int64_t p, double* __restrict__ row) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < K) row[j] = R[(int64_t)j * L + p];
}

// R -= q row^T
__global__ void k_rank1(int64_t L, int K, double* __restrict__ R, const double* __restrict__ q,
                        const double* __restrict__ row) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (l >= L) return;
    R[(int64_t)j * L + l] -= q[l] * row[j];
}

// ------------------------------------------------------------ host helpers
namespace {

// Symmetric eigendecomposition A = V diag(w) V^T of a dense n x n matrix
// (row-major in and out; column j of V the eigenvector of w[j]; unordered),
// the textbook two-phase method (Golub & Van Loan, "Matrix Computations",
// Sec. 8.3): Householder reduction T = Q^T A Q to tridiagonal form, Q
// accumulated from its reflectors, then implicit symmetric QR steps with the
// Wilkinson shift on T, each step a bulge chase of Givens rotations that are
// applied to the columns of Q as well.  ~8/3 n^3 flops for the reduction and
// the accumulation plus 6 n per Givens rotation (~6 n^3 in all); every inner
// loop runs along a row.  At a few thousand snapshots this is ~10x less work
// than cyclic Jacobi (~10 sweeps of ~6 n^3, with column access).
bool sym_eig(std::vector<double> A, int n, std::vector<double>& w, std::vector<double>& V) {
    auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
    std::vector<double> d(n), e(n, 0.0);        // diagonal, sub-diagonal e[i] = T(i+1, i)
    std::vector<std::vector<double>> hv(n > 2 ? n - 2 : 0);   // reflector vectors (v[0] = 1)
    std::vector<double> hb(n > 2 ? n - 2 : 0, 0.0);           // and their beta
    std::vector<double> p(n), q(n);
    // phase 1: for column k, a reflector P_k = I - beta v v^T maps A(k+1:n, k) to a multiple of e_1
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;                 // length of the trailing block
        std::vector<double>& v = hv[k];
        v.assign(m, 0.0);
        double sig = 0.0;
        for (int i = 1; i < m; ++i) {
            v[i] = a(k + 1 + i, k);
            sig += v[i] * v[i];
        }
        const double x0 = a(k + 1, k);
        double beta = 0.0, alpha = x0;           // alpha: the new sub-diagonal entry
        v[0] = 1.0;
        if (sig > 0.0) {
            const double mu = sqrt(x0 * x0 + sig);
            const double v0 = x0 <= 0.0 ? x0 - mu : -sig / (x0 + mu);   // cancellation-free x0 - mu
            beta = 2.0 * v0 * v0 / (sig + v0 * v0);
            for (int i = 1; i < m; ++i) v[i] /= v0;
            alpha = mu;
        }
        hb[k] = beta;
        e[k] = alpha;
        if (beta == 0.0) continue;
        // p = beta * B v, with B = A(k+1:n, k+1:n); q = p - (beta/2) (p.v) v; B -= v q^T + q v^T
        double pv = 0.0;
        for (int i = 0; i < m; ++i) {
            const double* row = &A[(size_t)(k + 1 + i) * n + k + 1];
            double acc = 0.0;
            for (int j = 0; j < m; ++j) acc += row[j] * v[j];
            p[i] = beta * acc;
            pv += p[i] * v[i];
        }
        for (int i = 0; i < m; ++i) q[i] = p[i] - 0.5 * beta * pv * v[i];
        for (int i = 0; i < m; ++i) {
            double* row = &A[(size_t)(k + 1 + i) * n + k + 1];
            const double vi = v[i], qi = q[i];
            for (int j = 0; j < m; ++j) row[j] -= vi * q[j] + qi * v[j];
        }
    }
    for (int i = 0; i < n; ++i) d[i] = a(i, i);
    if (n >= 2) e[n - 2] = a(n - 1, n - 2);
    // Q = P_0 P_1 ... P_{n-3}, kept transposed (row j of Qt = column j of Q) so
    // that both the accumulation and the rotations below stream along rows:
    // Qt = P_{n-3} ... P_0, built as Qt <- Qt P_k for k descending
    std::vector<double> Qt((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Qt[(size_t)i * n + i] = 1.0;
    for (int k = n - 3; k >= 0; --k) {
        const double beta = hb[k];
        if (beta == 0.0) continue;
        const std::vector<double>& v = hv[k];
        const int m = n - k - 1;
        for (int i = 0; i < m; ++i) {
            double* row = &Qt[(size_t)(k + 1 + i) * n + k + 1];
            double dot = 0.0;
            for (int j = 0; j < m; ++j) dot += row[j] * v[j];
            const double f = beta * dot;
            for (int j = 0; j < m; ++j) row[j] -= f * v[j];
        }
    }
    // phase 2: implicit QR with the Wilkinson shift on the unreduced trailing block [lo, hi]
    // an off-diagonal entry is negligible below eps times its diagonal
    // neighbours plus a floor of 1e-3 eps ||T|| (eigenvalues then carry an
    // absolute error of order eps ||A||, the backward-stable bound)
    const double eps = 2.220446049250313e-16;
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) tnorm = fmax(tnorm, fabs(d[i]) + (i ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0));
    int hi = n - 1, guard = 0;
    while (hi > 0 && guard < 64 * n) {
        for (int i = 0; i < hi; ++i)
            if (fabs(e[i]) <= eps * (fabs(d[i]) + fabs(d[i + 1]) + 1e-3 * tnorm)) e[i] = 0.0;
        while (hi > 0 && e[hi - 1] == 0.0) --hi;
        if (hi == 0) break;
        int lo = hi - 1;
        while (lo > 0 && e[lo - 1] != 0.0) --lo;
        ++guard;
        // Wilkinson shift: the eigenvalue of the trailing 2x2 block closer to d[hi]
        const double dd = 0.5 * (d[hi - 1] - d[hi]);
        const double e2 = e[hi - 1] * e[hi - 1];
        const double mu = d[hi] - e2 / (dd + (dd >= 0.0 ? 1.0 : -1.0) * hypot(dd, e[hi - 1]));
        // chase the bulge from (lo+1, lo) down to the end of the block
        double x = d[lo] - mu, z = e[lo];
        for (int k = lo; k < hi; ++k) {
            // Givens rotation G = [c s; -s c] with G^T [x; z] = [r; 0]
            const double r = hypot(x, z);
            const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? -z / r : 0.0;
            if (k > lo) e[k - 1] = r;
            // T <- G^T T G on rows/columns k, k+1
            const double dk = d[k], dk1 = d[k + 1], ek = e[k];
            d[k] = c * c * dk - 2.0 * c * s * ek + s * s * dk1;
            d[k + 1] = s * s * dk + 2.0 * c * s * ek + c * c * dk1;
            e[k] = c * s * (dk - dk1) + (c * c - s * s) * ek;
            if (k + 1 < hi) {
                x = e[k];
                z = -s * e[k + 1];           // the bulge at (k+2, k)
                e[k + 1] *= c;
            }
            // Q <- Q G on columns k, k+1, i.e. Qt <- G^T Qt on rows k, k+1
            double* rk = &Qt[(size_t)k * n];
            double* rk1 = &Qt[(size_t)(k + 1) * n];
            for (int i = 0; i < n; ++i) {
                const double vk = rk[i], vk1 = rk1[i];
                rk[i] = c * vk - s * vk1;
                rk1[i] = s * vk + c * vk1;
            }
        }
    }
    V.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) V[(size_t)i * n + j] = Qt[(size_t)j * n + i];
    w.swap(d);
    return hi == 0;
}

// lower Cholesky factor of a symmetric positive definite r x r matrix;
// returns the number of leading columns factored (r on success): a pivot
// below 1e-14 of its diagonal entry marks a numerically dependent mode
int cholesky(std::vector<double>& G, int r) {
    for (int j = 0; j < r; ++j) {
        double d = G[(size_t)j * r + j];
        const double d0 = d;
        for (int k = 0; k < j; ++k) d -= G[(size_t)j * r + k] * G[(size_t)j * r + k];
        if (!(d > 1e-14 * d0)) return j;
        d = sqrt(d);
        G[(size_t)j * r + j] = d;
        for (int i = j + 1; i < r; ++i) {
            double x = G[(size_t)i * r + j];
            for (int k = 0; k < j; ++k) x -= G[(size_t)i * r + k] * G[(size_t)j * r + k];
            G[(size_t)i * r + j] = x / d;
        }
        for (int k = j + 1; k < r; ++k) G[(size_t)j * r + k] = 0.0;
    }
    return r;
}

struct Dev {
    std::vector<void*> bufs;
    ~Dev() {
        for (void* p : bufs) cudaFree(p);
    }
    template <class T>
    T* alloc(size_t n) {
        void* p = nullptr;
        if (cudaMalloc(&p, sizeof(T) * (n ? n : 1)) != cudaSuccess) return nullptr;
        bufs.push_back(p);
        return static_cast<T*>(p);
    }
};

inline unsigned nbk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// D[:, k] = S[:, k] - S[:, 0]
__global__ void k_sub_first(int64_t L, int K, const double* __restrict__ S, double* __restrict__ D) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (l < L) D[(int64_t)k * L + l] = S[(int64_t)k * L + l] - S[l];
}

// W-orthonormal POD modes (column-major L x r on the device) of the snapshot
// block S (column-major L x K on the device, column 0 the initial state) with
// weights w (device, L): the initial state's direction first, then the POD
// modes of the snapshots' differences from it (the same span as the
// snapshots; the differences' Gram matrix resolves their singular values,
// which the large common part would push below the Gram route's precision).
static int pod_block(mb_cell* c, Dev& dv, int64_t L, int K, const double* S, const double* w, int rmax, double tol,
                     double** modes, int* r_out) {
    cudaStream_t s = c->stream;
    *r_out = 0;
    *modes = nullptr;
    if (L == 0 || K == 0 || rmax <= 0) return MB_OK;
    double* G = dv.alloc<double>((size_t)K * K);
    double* Dif = dv.alloc<double>((size_t)L * K);
    double* n0 = dv.alloc<double>(1);
    if (!G || !Dif || !n0) return MB_ENOMEM;
    dim3 gb((K + GT - 1) / GT, (K + GT - 1) / GT), tb(GT, GT);
    // is the initial state nonzero in this block?
    k_atwb<<<dim3(1, 1), tb, 0, s>>>(L, 1, 1, S, S, w, n0), count_launch(c);
    double h0 = 0.0;
    MB_CUDA(cudaMemcpyAsync(&h0, n0, 8, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    const bool anchor = h0 > 0.0;
    const double* S0 = S;   // column 0: the initial state
    if (anchor) {
        k_sub_first<<<dim3(nbk(L), K), 256, 0, s>>>(L, K, S, Dif), count_launch(c);
        S = Dif;
        rmax -= 1;
    }
    k_atwb<<<gb, tb, 0, s>>>(L, K, K, S, S, w, G), count_launch(c);
    std::vector<double> hG((size_t)K * K);
    MB_CUDA(cudaMemcpyAsync(hG.data(), G, 8 * hG.size(), cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    std::vector<double> ev, V;
    if (!sym_eig(hG, K, ev, V)) {
        set_error("mb_rom_build: symmetric eigensolver did not converge");
        return MB_EINVAL;
    }
    std::vector<int> order(K);
    for (int i = 0; i < K; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return ev[a] > ev[b]; });
    const double l1 = ev[order[0]];
    int rd = 0;
    if (l1 > 0)
        while (rd < rmax && rd < K && ev[order[rd]] > tol * tol * l1) ++rd;
    const int a0 = anchor ? 1 : 0;
    int r = rd + a0;
    if (r == 0) return MB_OK;
    std::vector<double> X((size_t)K * (rd ? rd : 1));
    for (int j = 0; j < rd; ++j) {
        const double sc = 1.0 / sqrt(ev[order[j]]);
        for (int k = 0; k < K; ++k) X[(size_t)k * rd + j] = V[(size_t)k * K + order[j]] * sc;
    }
    double* dX = dv.alloc<double>(X.size());
    double* Y = dv.alloc<double>((size_t)L * r);
    double* Y2 = dv.alloc<double>((size_t)L * r);
    double* Gm = dv.alloc<double>((size_t)r * r);
    if (!dX || !Y || !Y2 || !Gm) return MB_ENOMEM;
    if (anchor) MB_CUDA(cudaMemcpyAsync(Y, S0, 8 * L, cudaMemcpyDeviceToDevice, s));
    if (rd) {
        MB_CUDA(cudaMemcpyAsync(dX, X.data(), 8 * X.size(), cudaMemcpyHostToDevice, s));
        k_sx<<<dim3(nbk(L), rd), 256, 0, s>>>(L, K, rd, S, dX, Y + (size_t)a0 * L), count_launch(c);
    }
    // two Cholesky passes: Y <- Y L^-T with L L^T = Y^T W Y
    for (int pass = 0; pass < 2; ++pass) {
        dim3 gr((r + GT - 1) / GT, (r + GT - 1) / GT);
        k_atwb<<<gr, tb, 0, s>>>(L, r, r, Y, Y, w, Gm), count_launch(c);
        std::vector<double> hm((size_t)r * r);
        MB_CUDA(cudaMemcpyAsync(hm.data(), Gm, 8 * hm.size(), cudaMemcpyDeviceToHost, s));
        MB_CUDA(cudaStreamSynchronize(s));
        const int rk = cholesky(hm, r);
        if (rk < 1) {
            set_error("mb_rom_build: POD modes not independent");
            return MB_EINVAL;
        }
        if (rk < r) {
            // keep the leading rk modes (the columns of Y are ordered by singular value)
            std::vector<double> hk((size_t)rk * rk);
            for (int i = 0; i < rk; ++i)
                for (int j = 0; j < rk; ++j) hk[(size_t)i * rk + j] = hm[(size_t)i * r + j];
            hm.swap(hk);
            r = rk;
        }
        // Linv^T (r x r row-major): solve L Z = I, then X = Z^T
        std::vector<double> Z((size_t)r * r, 0.0);
        for (int col = 0; col < r; ++col)
            for (int i = 0; i < r; ++i) {
                double x = (i == col) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k) x -= hm[(size_t)i * r + k] * Z[(size_t)k * r + col];
                Z[(size_t)i * r + col] = x / hm[(size_t)i * r + i];
            }
        std::vector<double> Xt((size_t)r * r);
        for (int i = 0; i < r; ++i)
            for (int j = 0; j < r; ++j) Xt[(size_t)i * r + j] = Z[(size_t)j * r + i];
        double* dZ = dv.alloc<double>((size_t)r * r);
        if (!dZ) return MB_ENOMEM;
        MB_CUDA(cudaMemcpyAsync(dZ, Xt.data(), 8 * Xt.size(), cudaMemcpyHostToDevice, s));
        k_sx<<<dim3(nbk(L), r), 256, 0, s>>>(L, r, r, Y, dZ, Y2), count_launch(c);
        std::swap(Y, Y2);
    }
    *modes = Y;
    *r_out = r;
    MB_CUDA_LAUNCH("pod");
    return MB_OK;
}

// EI-Greedy on the training columns T (column-major L x K, overwritten by the
// residuals): basis Q (host, column-major L x m) and points P (host, m)
static int ei_greedy(mb_cell* c, Dev& dv, int64_t L, int K, double* T, int mmax, double tol, std::vector<double>& Q,
                     std::vector<int64_t>& P) {
    cudaStream_t s = c->stream;
    Q.clear();
    P.clear();
    if (K == 0 || mmax <= 0) return MB_OK;
    double* cm = dv.alloc<double>(K);
    double* q = dv.alloc<double>(L);
    double* row = dv.alloc<double>(K);
    int64_t* pi = dv.alloc<int64_t>(1);
    if (!cm || !q || !row || !pi) return MB_ENOMEM;
    std::vector<double> hcm(K);
    double scale = -1.0;
    for (int m = 0; m < mmax; ++m) {
        k_colmax<<<K, 256, 0, s>>>(L, T, cm), count_launch(c);
        MB_CUDA(cudaMemcpyAsync(hcm.data(), cm, 8 * K, cudaMemcpyDeviceToHost, s));
        MB_CUDA(cudaStreamSynchronize(s));
        int k = 0;
        for (int j = 1; j < K; ++j)
            if (hcm[j] > hcm[k]) k = j;
        if (scale < 0) scale = hcm[k];
        if (!(hcm[k] > tol * scale) || hcm[k] == 0.0) break;
        k_argmax<<<1, 256, 0, s>>>(L, T + (int64_t)k * L, pi), count_launch(c);
        int64_t p = 0;
        MB_CUDA(cudaMemcpyAsync(&p, pi, 8, cudaMemcpyDeviceToHost, s));
        MB_CUDA(cudaStreamSynchronize(s));
        k_ei_newvec<<<nbk(L), 256, 0, s>>>(L, T, k, p, q), count_launch(c);
        k_getrow<<<nbk(K), 256, 0, s>>>(L, K, T, p, row), count_launch(c);
        k_rank1<<<dim3(nbk(L), K), 256, 0, s>>>(L, K, T, q, row), count_launch(c);
        size_t o = Q.size();
        Q.resize(o + (size_t)L);
        MB_CUDA(cudaMemcpyAsync(Q.data() + o, q, 8 * L, cudaMemcpyDeviceToHost, s));
        P.push_back(p);
    }
    MB_CUDA(cudaStreamSynchronize(s));
    MB_CUDA_LAUNCH("ei_greedy");
    return MB_OK;
}

}  // namespace mb

using namespace mb;

static bool build_opts_ok(const mb_rom_build_opts* o) {
    return o && o->n_params >= 1 && o->params && o->dt > 0 && o->n_steps >= 1 && o->n_c >= 0 && o->n_n >= 0 &&
           o->n_phi >= 0 && o->m_bv >= 0 && o->m_1c >= 0 && o->n_c + o->n_n + o->n_phi >= 1;
}

// 1. snapshots: every Newton stage of n_steps steps at each parameter point,
// from the cell's current state (restored afterwards), with its gates
static int collect_snapshots(mb_cell* c, const mb_rom_build_opts* o, std::vector<double>& u_init,
                             std::vector<std::vector<double>>& su, std::vector<std::vector<uint8_t>>& sg) {
    const int64_t N = c->D.N, F = c->D.F, n = c->n;
    cudaStream_t s = c->stream;
    u_init.resize(n);
    MB_CUDA(cudaMemcpy(u_init.data(), c->u, 8 * n, cudaMemcpyDeviceToHost));
    const double s0 = c->s_i0, k0 = c->k_pl;
    int rc = MB_OK;
    {
        // gates at the initial state (rule of the step)
        su.push_back(u_init);
        sg.emplace_back(F);
        if (F) {
            MB_CUDA(cudaMemcpyAsync(c->u_old, c->u, 8 * n, cudaMemcpyDeviceToDevice, s));
            rc = launch_gate(c, c->u_old, c->u_old + 2 * N, c->gate2, s);
            if (rc) return rc;
            MB_CUDA(cudaMemcpyAsync(sg.back().data(), c->gate2, F, cudaMemcpyDeviceToHost, s));
            MB_CUDA(cudaStreamSynchronize(s));
        }
    }
    c->snap_u = &su;
    c->snap_g = &sg;
    for (int ip = 0; ip < o->n_params && rc == MB_OK; ++ip) {
        MB_CUDA(cudaMemcpy(c->u, u_init.data(), 8 * n, cudaMemcpyHostToDevice));
        c->s_i0 = o->params[ip].s_i0;
        c->k_pl = o->params[ip].k_pl;
        for (int k = 0; k < o->n_steps && rc == MB_OK; ++k) {
            mb_step_info info;
            rc = newton_step(c, o->dt, o->params[ip].I_app, &info);
        }
    }
    c->snap_u = nullptr;
    c->snap_g = nullptr;
    c->s_i0 = s0;
    c->k_pl = k0;
    c->has_hist = false;
    MB_CUDA(cudaMemcpy(c->u, u_init.data(), 8 * n, cudaMemcpyHostToDevice));
    return rc;
}

// 2.-4. POD, EI-Greedy and projections from the snapshots; dims (may be
// NULL) receive the sizes taken: modes of c, n, phi, then the two numbers of
// points
static int rom_from_snapshots(mb_cell* c, const mb_rom_build_opts* o, const std::vector<double>& u_init,
                              const std::vector<std::vector<double>>& su, const std::vector<std::vector<uint8_t>>& sg,
                              mb_rom** out, int* dims) {
    const int64_t N = c->D.N, F = c->D.F, n = c->n;
    cudaStream_t s = c->stream;
    int rc = MB_OK;
    const int K = (int)su.size();
    Dev dv;
    // snapshot blocks, column-major
    double* Sc = dv.alloc<double>((size_t)N * K);
    double* Sp = dv.alloc<double>((size_t)N * K);
    double* Sn = dv.alloc<double>((size_t)(F ? F : 1) * K);
    double* Sall = dv.alloc<double>((size_t)n * K);
    uint8_t* Gall = dv.alloc<uint8_t>((size_t)(F ? F : 1) * K);
    double* wv = dv.alloc<double>(N);
    double* wf = dv.alloc<double>(F ? F : 1);
    if (!Sc || !Sp || !Sn || !Sall || !Gall || !wv || !wf) { set_error("mb_rom_build: device memory"); return MB_ENOMEM; }
    for (int k = 0; k < K; ++k) {
        MB_CUDA(cudaMemcpyAsync(Sall + (size_t)k * n, su[k].data(), 8 * n, cudaMemcpyHostToDevice, s));
        MB_CUDA(cudaMemcpyAsync(Sc + (size_t)k * N, su[k].data(), 8 * N, cudaMemcpyHostToDevice, s));
        MB_CUDA(cudaMemcpyAsync(Sp + (size_t)k * N, su[k].data() + N, 8 * N, cudaMemcpyHostToDevice, s));
        if (F) {
            MB_CUDA(cudaMemcpyAsync(Sn + (size_t)k * F, su[k].data() + 2 * N, 8 * F, cudaMemcpyHostToDevice, s));
            MB_CUDA(cudaMemcpyAsync(Gall + (size_t)k * F, sg[k].data(), F, cudaMemcpyHostToDevice, s));
        }
    }
    {
        std::vector<double> hw(N, c->P.V), hf(F ? F : 1, c->P.A);
        MB_CUDA(cudaMemcpyAsync(wv, hw.data(), 8 * N, cudaMemcpyHostToDevice, s));
        MB_CUDA(cudaMemcpyAsync(wf, hf.data(), 8 * hf.size(), cudaMemcpyHostToDevice, s));
        MB_CUDA(cudaStreamSynchronize(s));
    }
    // --- 2. POD of c, n, phi
    double *Mc = nullptr, *Mn = nullptr, *Mp = nullptr;
    int rcn = 0, rnn = 0, rpn = 0;
    if ((rc = pod_block(c, dv, N, K, Sc, wv, o->n_c, o->pod_tol, &Mc, &rcn))) return rc;
    if (F && (rc = pod_block(c, dv, F, K, Sn, wf, o->n_n, o->pod_tol, &Mn, &rnn))) return rc;
    if ((rc = pod_block(c, dv, N, K, Sp, wv, o->n_phi, o->pod_tol, &Mp, &rpn))) return rc;
    const int Nr = rcn + rnn + rpn;
    if (Nr < 1) { set_error("mb_rom_build: empty reduced basis"); return MB_EINVAL; }
    // full-layout basis U (column-major n x Nr, device) and host row-major copy
    double* U = dv.alloc<double>((size_t)n * Nr);
    if (!U) return MB_ENOMEM;
    MB_CUDA(cudaMemsetAsync(U, 0, 8 * (size_t)n * Nr, s));
    for (int j = 0; j < rcn; ++j) MB_CUDA(cudaMemcpyAsync(U + (size_t)j * n, Mc + (size_t)j * N, 8 * N, cudaMemcpyDeviceToDevice, s));
    for (int j = 0; j < rnn; ++j)
        MB_CUDA(cudaMemcpyAsync(U + (size_t)(rcn + j) * n + 2 * N, Mn + (size_t)j * F, 8 * F, cudaMemcpyDeviceToDevice, s));
    for (int j = 0; j < rpn; ++j)
        MB_CUDA(cudaMemcpyAsync(U + (size_t)(rcn + rnn + j) * n + N, Mp + (size_t)j * N, 8 * N, cudaMemcpyDeviceToDevice, s));
    // --- 3. EI training columns
    const int Kbv = 3 * K;
    double* Tbv = dv.alloc<double>((size_t)n * Kbv);
    double* T1c = dv.alloc<double>((size_t)n * K);
    if (!Tbv || !T1c) { set_error("mb_rom_build: device memory"); return MB_ENOMEM; }
    MB_CUDA(cudaMemsetAsync(Tbv, 0, 8 * (size_t)n * Kbv, s));
    MB_CUDA(cudaMemsetAsync(T1c, 0, 8 * (size_t)n * K, s));
    for (int k = 0; k < K; ++k) {
        double* ob = Tbv + (size_t)(3 * k) * n;
        k_subops<<<nbk(N), 256, 0, s>>>(c->P, c->D, c->vcode, Sall + (size_t)k * n, Gall + (size_t)k * (F ? F : 1), ob,
                                        ob + n, ob + 2 * n, T1c + (size_t)k * n), count_launch(c);
    }
    MB_CUDA_LAUNCH("subops");
    // drop all-zero training columns
    auto compact = [&](double* T, int cols, int* kept) -> int {
        double* cm = dv.alloc<double>(cols);
        if (!cm) return MB_ENOMEM;
        k_colmax<<<cols, 256, 0, s>>>(n, T, cm), count_launch(c);
        std::vector<double> h(cols);
        MB_CUDA(cudaMemcpyAsync(h.data(), cm, 8 * cols, cudaMemcpyDeviceToHost, s));
        MB_CUDA(cudaStreamSynchronize(s));
        int m = 0;
        for (int j = 0; j < cols; ++j) {
            if (h[j] == 0.0) continue;
            if (m != j) MB_CUDA(cudaMemcpyAsync(T + (size_t)m * n, T + (size_t)j * n, 8 * n, cudaMemcpyDeviceToDevice, s));
            ++m;
        }
        *kept = m;
        return MB_OK;
    };
    int kb = 0, k1 = 0;
    if ((rc = compact(Tbv, Kbv, &kb)) || (rc = compact(T1c, K, &k1))) return rc;
    std::vector<double> Qbv, Q1c;
    std::vector<int64_t> Pbv, P1c;
    if ((rc = ei_greedy(c, dv, n, kb, Tbv, o->m_bv, o->ei_tol, Qbv, Pbv))) return rc;
    if ((rc = ei_greedy(c, dv, n, k1, T1c, o->m_1c, o->ei_tol, Q1c, P1c))) return rc;
    const int Mb = (int)Pbv.size(), M1 = (int)P1c.size();
    // --- 4. projections; D = row weights (1 on c and phi rows, A on face rows)
    std::vector<double> hD(n, 1.0), hDMs(n, 0.0), hbnd(n, 0.0);
    std::vector<uint32_t> hvc(N);
    MB_CUDA(cudaMemcpy(hvc.data(), c->vcode, 4 * N, cudaMemcpyDeviceToHost));
    for (int64_t i = 2 * N; i < n; ++i) { hD[i] = c->P.A; hDMs[i] = c->P.A; }
    for (int64_t v = 0; v < N; ++v)
        if (has_c(vc_phase(hvc[v]))) hDMs[v] = c->P.V;
    const int64_t last0 = (int64_t)(c->D.nt - 1) * c->D.syz;
    for (int64_t v = last0; v < N; ++v)
        if (vc_phase(hvc[v]) == PCP) hbnd[N + v] = c->P.A;
    double* dD = dv.alloc<double>(n);
    double* dDMs = dv.alloc<double>(n);
    double* LU = dv.alloc<double>((size_t)n * Nr);
    double* dMs = dv.alloc<double>((size_t)Nr * Nr);
    double* dAl = dv.alloc<double>((size_t)Nr * Nr);
    double* dbnd = dv.alloc<double>(n);
    double* dbb = dv.alloc<double>(Nr);
    if (!dD || !dDMs || !LU || !dMs || !dAl || !dbnd || !dbb) return MB_ENOMEM;
    MB_CUDA(cudaMemcpyAsync(dD, hD.data(), 8 * n, cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemcpyAsync(dDMs, hDMs.data(), 8 * n, cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemcpyAsync(dbnd, hbnd.data(), 8 * n, cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemsetAsync(LU, 0, 8 * (size_t)n * Nr, s));
    for (int j = 0; j < Nr; ++j) k_lin_apply<<<nbk(N), 256, 0, s>>>(c->P, c->D, c->vcode, U + (size_t)j * n, LU + (size_t)j * n), count_launch(c);
    const dim3 tb(GT, GT), gr((Nr + GT - 1) / GT, (Nr + GT - 1) / GT);
    k_atwb<<<gr, tb, 0, s>>>(n, Nr, Nr, U, U, dDMs, dMs), count_launch(c);
    k_atwb<<<gr, tb, 0, s>>>(n, Nr, Nr, U, LU, dD, dAl), count_launch(c);
    k_atwb<<<dim3(1, (Nr + GT - 1) / GT), tb, 0, s>>>(n, Nr, 1, U, dbnd, dD, dbb), count_launch(c);
    auto project_ei = [&](const std::vector<double>& Q, const std::vector<int64_t>& P, std::vector<double>& out) -> int {
        const int M = (int)P.size();
        out.assign((size_t)Nr * M, 0.0);
        if (!M) return MB_OK;
        double* dQ = dv.alloc<double>((size_t)n * M);
        double* dY = dv.alloc<double>((size_t)Nr * M);
        if (!dQ || !dY) return MB_ENOMEM;
        MB_CUDA(cudaMemcpyAsync(dQ, Q.data(), 8 * Q.size(), cudaMemcpyHostToDevice, s));
        k_atwb<<<dim3((M + GT - 1) / GT, (Nr + GT - 1) / GT), tb, 0, s>>>(n, Nr, M, U, dQ, dD, dY), count_launch(c);
        std::vector<double> Y((size_t)Nr * M);
        MB_CUDA(cudaMemcpyAsync(Y.data(), dY, 8 * Y.size(), cudaMemcpyDeviceToHost, s));
        MB_CUDA(cudaStreamSynchronize(s));
        // X Q_P = Y with Q_P = Q[P, :] unit lower triangular: columns from the last
        for (int i = 0; i < Nr; ++i)
            for (int j = M - 1; j >= 0; --j) {
                double x = Y[(size_t)i * M + j];
                for (int k = j + 1; k < M; ++k) x -= out[(size_t)i * M + k] * Q[(size_t)j * n + P[k]];
                out[(size_t)i * M + j] = x;
            }
        return MB_OK;
    };
    std::vector<double> Pb, P1;
    if ((rc = project_ei(Qbv, Pbv, Pb)) || (rc = project_ei(Q1c, P1c, P1))) return rc;
    // host copies of U (row-major), Ms, Alin, bbnd
    std::vector<double> Uc((size_t)n * Nr), Ur((size_t)n * Nr), Ms((size_t)Nr * Nr), Al((size_t)Nr * Nr), bb(Nr);
    MB_CUDA(cudaMemcpyAsync(Uc.data(), U, 8 * Uc.size(), cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaMemcpyAsync(Ms.data(), dMs, 8 * Ms.size(), cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaMemcpyAsync(Al.data(), dAl, 8 * Al.size(), cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaMemcpyAsync(bb.data(), dbb, 8 * bb.size(), cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < Nr; ++j) Ur[(size_t)i * Nr + j] = Uc[(size_t)j * n + i];
    // output functionals and initial coefficients
    std::vector<double> scp(Nr, 0.0), sac(Nr, 0.0), a0(Nr, 0.0);
    int64_t nlast = 0, nG = 0;
    for (int64_t v = last0; v < N; ++v) ++nlast;
    for (int64_t v = 0; v < N; ++v) nG += vc_phase(hvc[v]) == PG;
    for (int j = 0; j < Nr; ++j) {
        double a = 0.0, g = 0.0, p = 0.0;
        for (int64_t v = last0; v < N; ++v) a += Ur[(size_t)(N + v) * Nr + j];
        for (int64_t v = 0; v < N; ++v)
            if (vc_phase(hvc[v]) == PG) g += Ur[(size_t)v * Nr + j];
        for (int64_t i = 0; i < n; ++i) p += Ur[(size_t)i * Nr + j] * (i >= 2 * N ? c->P.A : c->P.V) * u_init[i];
        scp[j] = nlast ? a / nlast : 0.0;
        sac[j] = nG ? g / nG : 0.0;
        a0[j] = p;
    }
    mb_rom_data d{Nr, Mb, M1, Ur.data(), Pbv.data(), P1c.data(), Ms.data(), Al.data(), bb.data(), Pb.data(),
                  P1.data(), scp.data(), sac.data(), a0.data()};
    if (dims) {
        dims[0] = rcn; dims[1] = rnn; dims[2] = rpn; dims[3] = Mb; dims[4] = M1;
    }
    return mb_rom_create(c, &d, out);
}

extern "C" int mb_rom_build(mb_cell* c, const mb_rom_build_opts* o, mb_rom** out) {
    if (!c || !out || !build_opts_ok(o)) {
        set_error("mb_rom_build: invalid argument");
        return MB_EINVAL;
    }
    std::vector<double> u_init;
    std::vector<std::vector<double>> su;
    std::vector<std::vector<uint8_t>> sg;
    int rc = collect_snapshots(c, o, u_init, su, sg);
    if (rc) return rc;
    return rom_from_snapshots(c, o, u_init, su, sg, out, nullptr);
}

extern "C" int mb_rom_build_pair(mb_cell* c, const mb_rom_build_opts* o, double frac, mb_rom** rom,
                                 mb_rom** rom_val) {
    if (!c || !rom || !rom_val || !build_opts_ok(o) || !(frac > 0.0 && frac <= 1.0)) {
        set_error("mb_rom_build_pair: invalid argument");
        return MB_EINVAL;
    }
    std::vector<double> u_init;
    std::vector<std::vector<double>> su;
    std::vector<std::vector<uint8_t>> sg;
    int rc = collect_snapshots(c, o, u_init, su, sg);
    if (rc) return rc;
    int dims[5];
    if ((rc = rom_from_snapshots(c, o, u_init, su, sg, rom_val, dims))) return rc;
    // the reduced model: ceil(frac x) of the validation model's modes per block and points per basis
    mb_rom_build_opts o2 = *o;
    auto part = [&](int x) { return (int)ceil(frac * (double)x - 1e-9); };
    o2.n_c = part(dims[0]);
    o2.n_n = part(dims[1]);
    o2.n_phi = part(dims[2]);
    o2.m_bv = part(dims[3]);
    o2.m_1c = part(dims[4]);
    if ((rc = rom_from_snapshots(c, &o2, u_init, su, sg, rom, nullptr))) {
        mb_rom_destroy(*rom_val);
        *rom_val = nullptr;
        return rc;
    }
    return MB_OK;
}

// ------------------------------------------------------------ test hooks
extern "C" int mb_debug_symeig(int n, const double* A, double* w, double* V) {
    if (n < 1 || !A || !w || !V) { set_error("mb_debug_symeig: invalid argument"); return MB_EINVAL; }
    std::vector<double> a(A, A + (size_t)n * n), ww, vv;
    if (!sym_eig(a, n, ww, vv)) { set_error("mb_debug_symeig: no convergence"); return MB_EINVAL; }
    memcpy(w, ww.data(), sizeof(double) * n);
    memcpy(V, vv.data(), sizeof(double) * (size_t)n * n);
    return MB_OK;
}
