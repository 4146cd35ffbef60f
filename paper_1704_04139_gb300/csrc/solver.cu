// solver.cu -- Newton-Krylov driver of one implicit Euler step (Eq.
// ap4:detailed): scaled right-preconditioned flexible GMRES with classical
// Gram-Schmidt and one re-orthogonalisation, the damped Newton update, the
// plating active-set passes and step halving on failure.
// Precision: the state and the Newton residual are FP64; the Krylov solver
// works in FP32 arithmetic with an FP32 basis V and float-float (hi + lo)
// preconditioned directions Z and solution x, whose large near-null
// components must keep their small structure; dot products use FP32 products
// and FP64 sums (deterministic order).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "mb_internal.h"
#include "mb_reduce.cuh"

namespace mb {

// MB_DEBUG=1 in the environment prints one line per Newton iteration to stderr.
int debug_level() {
    static int lvl = -1;
    if (lvl < 0) {
        const char* e = getenv("MB_DEBUG");
        lvl = e ? atoi(e) : 0;
    }
    return lvl;
}

constexpr int MDOT_G = 8;   // dot products per launch

struct HParam {
    float h[64];
};
struct HParamDF {
    float2 y[64];
};

struct Krylov {
    int m = 0;
    int64_t n = 0;
    float* V = nullptr;      // (m+1) x n
    float2* Z = nullptr;     // m x n
    float* w = nullptr;      // n
    float* b = nullptr;      // n  right-hand side (scaled, row-equilibrated)
    float2* x = nullptr;     // n  solution (scaled)
};

// ------------------------------------------------------------ vector kernels
__global__ void __launch_bounds__(RED_THREADS)
k_mdot(const float* __restrict__ V, int64_t stride, int cnt, const float* __restrict__ w, int64_t n,
       double* partials) {
    float a32[MDOT_G];
#pragma unroll
    for (int j = 0; j < MDOT_G; ++j) a32[j] = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float wi = w[i];
#pragma unroll
        for (int j = 0; j < MDOT_G; ++j)
            if (j < cnt) a32[j] = fmaf(V[j * stride + i], wi, a32[j]);
    }
    block_reduce_store_f32<MDOT_G>(a32, partials);
}

// w += sign * sum_j h[j] V_j
__global__ void k_mupdate(const float* __restrict__ V, int64_t stride, int cnt, HParam hp, float* __restrict__ w,
                          int64_t n, float sign) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc = 0.f;
    for (int j = 0; j < cnt; ++j) acc = fmaf(hp.h[j], V[j * stride + i], acc);
    w[i] = fmaf(sign, acc, w[i]);
}

// w -= sum_j h[j] V_j (as k_mupdate with sign -1), then the block partials
// of the updated w against V_j, j < cnt <= MDOT_G (NORM: against itself), in
// the grid and summation order of k_mdot: one pass of classical Gram-Schmidt
// fused with the products that follow it
template <bool NORM>
__global__ void __launch_bounds__(RED_THREADS)
k_mupd_dot(const float* __restrict__ V, int64_t stride, int cnt, HParam hp, float* __restrict__ w, int64_t n,
           double* partials) {
    constexpr int K = NORM ? 1 : MDOT_G;
    float a32[K];
#pragma unroll
    for (int j = 0; j < K; ++j) a32[j] = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float v[MDOT_G];
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < MDOT_G; ++j)
            if (j < cnt) {
                v[j] = V[j * stride + i];
                acc = fmaf(hp.h[j], v[j], acc);
            }
        const float wi = fmaf(-1.f, acc, w[i]);
        w[i] = wi;
        if (NORM) {
            a32[0] = fmaf(wi, wi, a32[0]);
        } else {
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (j < cnt) a32[j] = fmaf(v[j], wi, a32[j]);
        }
    }
    block_reduce_store_f32<K>(a32, partials);
}

// x += sum_j y[j] Z_j in float-float arithmetic
__global__ void k_combine(const float2* __restrict__ Z, int64_t stride, int cnt, HParamDF hp,
                          float2* __restrict__ x, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float2 acc = x[i];
    for (int j = 0; j < cnt; ++j) acc = df_add(acc, df_mul(Z[j * stride + i], hp.y[j]));
    x[i] = acc;
}

__global__ void k_scale(const float* __restrict__ a, float alpha, float* __restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = alpha * a[i];
}

// w = b - w
__global__ void k_rsub(const float* __restrict__ b, float* __restrict__ w, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = b[i] - w[i];
}

template <class A, class B>
__global__ void k_convert(const A* __restrict__ a, B* __restrict__ b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (B)a[i];
}

__global__ void k_axpy_d(double alpha, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += alpha * x[i];
}

// b_hat = -R / s_r / |diag|  (row-equilibrated right-hand side; is = 1/s_r).
// R is rounded to FP32 before the scaling (the right-hand side is FP32 either
// way; one FP64 conversion per element instead of a multiply and a conversion
// on GB300's narrow FP64 pipe); the per-phase scales from shared memory.
__global__ void k_scale_rhs(Dims D, const uint32_t* __restrict__ vc, const double* __restrict__ R, InvScales is,
                            const float* __restrict__ rowinv, float* __restrict__ b) {
    __shared__ float s_c[6];
    if (threadIdx.x < 6) s_c[threadIdx.x] = (float)is.c[threadIdx.x];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n = 2 * D.N + D.F;
    if (i >= n) return;
    float s;
    if (i < D.N) s = s_c[vc_phase(vc[i])];
    else if (i < 2 * D.N) s = (float)is.phi;
    else s = (float)is.n;
    b[i] = -(float)R[i] * s * rowinv[i];
}

// delta = s_u * x_hat (per-phase scales from shared memory)
__global__ void k_unscale(DevParams P, Dims D, const uint32_t* __restrict__ vc, const float2* __restrict__ x,
                          double* __restrict__ d) {
    __shared__ double s_c[6];
    if (threadIdx.x < 6) s_c[threadIdx.x] = P.cref[threadIdx.x];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n = 2 * D.N + D.F;
    if (i >= n) return;
    if (i < D.N) d[i] = s_c[vc_phase(vc[i])] * df_to_double(x[i]);
    else if (i < 2 * D.N) d[i] = df_to_double(x[i]);
    else d[i] = P.nc * df_to_double(x[i]);
}

static inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

// dots out[j] = <V_j, w> for j in [0, cnt)
static int mdot(mb_cell* c, const float* V, int64_t stride, int cnt, const float* w, int64_t n, double* out) {
    cudaStream_t s = c->stream;
    for (int j0 = 0; j0 < cnt; j0 += MDOT_G) {
        int k = cnt - j0 < MDOT_G ? cnt - j0 : MDOT_G;
        k_mdot<<<RED_BLOCKS, RED_THREADS, 0, s>>>(V + j0 * stride, stride, k, w, n, c->red), ::mb::count_launch(c);
        k_reduce_final<false><<<k, RED_THREADS, 0, s>>>(c->red, k, c->red_out + j0), ::mb::count_launch(c);
    }
    MB_CUDA_LAUNCH("mdot");
    MB_CUDA(cudaMemcpyAsync(c->h_red, c->red_out, 8 * cnt, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    memcpy(out, c->h_red, 8 * cnt);
    return MB_OK;
}

// w -= sum_j h[j] V_j, then out[j] = <V_j, w> (j < cnt) or, norm, out[0] = <w, w>;
// cnt <= MDOT_G
static int mupdate_dot(mb_cell* c, const float* V, int64_t stride, int cnt, const double* h, float* w, int64_t n,
                       bool norm, double* out) {
    cudaStream_t s = c->stream;
    HParam hp;
    for (int j = 0; j < cnt; ++j) hp.h[j] = (float)h[j];
    const int k = norm ? 1 : cnt;
    if (norm)
        k_mupd_dot<true><<<RED_BLOCKS, RED_THREADS, 0, s>>>(V, stride, cnt, hp, w, n, c->red), ::mb::count_launch(c);
    else
        k_mupd_dot<false><<<RED_BLOCKS, RED_THREADS, 0, s>>>(V, stride, cnt, hp, w, n, c->red), ::mb::count_launch(c);
    k_reduce_final<false><<<k, RED_THREADS, 0, s>>>(c->red, k, c->red_out), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("mupdate_dot");
    MB_CUDA(cudaMemcpyAsync(c->h_red, c->red_out, 8 * k, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    memcpy(out, c->h_red, 8 * k);
    return MB_OK;
}

static int mupdate(mb_cell* c, const float* V, int64_t stride, int cnt, const double* h, float* w, int64_t n,
                   float sign) {
    for (int j0 = 0; j0 < cnt; j0 += 64) {
        int k = cnt - j0 < 64 ? cnt - j0 : 64;
        HParam hp;
        for (int j = 0; j < k; ++j) hp.h[j] = (float)h[j0 + j];
        k_mupdate<<<nblk(n), 256, 0, c->stream>>>(V + j0 * stride, stride, k, hp, w, n, sign), ::mb::count_launch(c);
    }
    MB_CUDA_LAUNCH("mupdate");
    return MB_OK;
}

// Krylov operator: the row-equilibrated scaled JVP at the current Newton
// iterate, FP32 arithmetic on a float-float direction, from the interface
// partials stored by launch_lin_setup (evaluated from the FP64 state in FP64
// for MB_PREC_FP64, from its FP32 copy in FP32 for MB_PREC_MIXED).
struct OpCtx {
    const float* u32;
    const uint8_t* gate;
    double dt;
};

static int apply_op(mb_cell* c, const OpCtx& o, const float2* x, float* y) {
    (void)o;
    return launch_jvp_lin(c, x, y, c->stream);
}

// Flexible GMRES(m) on A x = b (x starts at zero), stopping at
// ||b - A x||_2 <= rtol ||b||_2 or after maxit iterations.
static int fgmres(mb_cell* c, Krylov* K, const OpCtx& o, double rtol, int maxit, int* its_out,
                  double* relres_out) {
    const int64_t n = K->n;
    const int m = K->m;
    cudaStream_t s = c->stream;
    std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m), hv(m + 1), h2(m + 1);
    MB_CUDA(cudaMemsetAsync(K->x, 0, n * sizeof(float2), s));
    double beta0 = 0.0;
    {
        double d;
        int rc = mdot(c, K->b, 0, 1, K->b, n, &d);
        if (rc) return rc;
        beta0 = sqrt(d);
    }
    *its_out = 0;
    *relres_out = 0.0;
    if (beta0 == 0.0) return MB_OK;
    if (!(beta0 == beta0)) { set_error("non-finite Newton residual"); return MB_ENOCONV; }
    int its = 0;
    double relres = 1.0;
    bool first = true;
    while (its < maxit) {
        // r = b - A x  (first cycle: r = b)
        double beta;
        const float* r0 = K->b;
        if (first) {
            beta = beta0;
        } else {
            int rc = apply_op(c, o, K->x, K->w);
            if (rc) return rc;
            k_rsub<<<nblk(n), 256, 0, s>>>(K->b, K->w, n), ::mb::count_launch(c);
            double d;
            rc = mdot(c, K->w, 0, 1, K->w, n, &d);
            if (rc) return rc;
            beta = sqrt(d);
            r0 = K->w;
        }
        first = false;
        k_scale<<<nblk(n), 256, 0, s>>>(r0, (float)(1.0 / beta), K->V, n), ::mb::count_launch(c);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        for (; j < m && its < maxit; ++j) {
            float* Vj = K->V + j * n;
            float2* Zj = K->Z + j * n;
            int rc = precond_apply(c, o.u32, o.gate, o.dt, Vj, Zj);
            if (rc) return rc;
            rc = apply_op(c, o, Zj, K->w);
            if (rc) return rc;
            // CGS2 (for up to MDOT_G basis vectors each update fused with the products after it)
            rc = mdot(c, K->V, n, j + 1, K->w, n, hv.data());
            if (rc) return rc;
            double d;
            if (j + 1 <= MDOT_G) {
                rc = mupdate_dot(c, K->V, n, j + 1, hv.data(), K->w, n, false, h2.data());
                if (rc) return rc;
                rc = mupdate_dot(c, K->V, n, j + 1, h2.data(), K->w, n, true, &d);
                if (rc) return rc;
            } else {
                rc = mupdate(c, K->V, n, j + 1, hv.data(), K->w, n, -1.f);
                if (rc) return rc;
                rc = mdot(c, K->V, n, j + 1, K->w, n, h2.data());
                if (rc) return rc;
                rc = mupdate(c, K->V, n, j + 1, h2.data(), K->w, n, -1.f);
                if (rc) return rc;
                rc = mdot(c, K->w, 0, 1, K->w, n, &d);
                if (rc) return rc;
            }
            for (int i = 0; i <= j; ++i) hv[i] += h2[i];
            double hn = sqrt(d);
            hv[j + 1] = hn;
            if (hn > 0) k_scale<<<nblk(n), 256, 0, s>>>(K->w, (float)(1.0 / hn), K->V + (j + 1) * n, n), ::mb::count_launch(c);
            // Givens rotations
            for (int i = 0; i < j; ++i) {
                double a = cs[i] * hv[i] + sn[i] * hv[i + 1];
                double b = -sn[i] * hv[i] + cs[i] * hv[i + 1];
                hv[i] = a; hv[i + 1] = b;
            }
            double den = sqrt(hv[j] * hv[j] + hv[j + 1] * hv[j + 1]);
            cs[j] = den > 0 ? hv[j] / den : 1.0;
            sn[j] = den > 0 ? hv[j + 1] / den : 0.0;
            hv[j] = den;
            hv[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; ++i) H[i * m + j] = hv[i];
            ++its;
            relres = fabs(g[j + 1]) / beta0;
            if (!(relres == relres)) { set_error("non-finite Krylov residual"); return MB_ENOCONV; }
            if (relres <= rtol || hn == 0.0) { ++j; break; }
        }
        // back substitution and x += Z y
        int k = j;
        for (int i = k - 1; i >= 0; --i) {
            double acc = g[i];
            for (int l = i + 1; l < k; ++l) acc -= H[i * m + l] * y[l];
            y[i] = acc / H[i * m + i];
        }
        for (int j0 = 0; j0 < k; j0 += 64) {
            int kk = k - j0 < 64 ? k - j0 : 64;
            HParamDF hp;
            for (int jj = 0; jj < kk; ++jj) {
                float yh = (float)y[j0 + jj];
                hp.y[jj] = make_float2(yh, (float)(y[j0 + jj] - (double)yh));
            }
            k_combine<<<nblk(n), 256, 0, s>>>(K->Z + j0 * n, n, kk, hp, K->x, n), ::mb::count_launch(c);
        }
        MB_CUDA_LAUNCH("fgmres update");
        if (relres <= rtol) break;
    }
    *its_out = its;
    *relres_out = relres;
    return MB_OK;
}

static int krylov_create(mb_cell* c, Krylov** out) {
    Krylov* K = new Krylov();
    K->m = c->opt.gmres_m;
    K->n = c->n;
    size_t n = (size_t)c->n;
    K->V = (float*)cell_alloc(c, 4 * n * (K->m + 1));
    K->Z = (float2*)cell_alloc(c, 8 * n * K->m);
    K->w = (float*)cell_alloc(c, 4 * n);
    K->b = (float*)cell_alloc(c, 4 * n);
    K->x = (float2*)cell_alloc(c, 8 * n);
    *out = K;
    if (!K->V || !K->Z || !K->w || !K->b || !K->x) return MB_ENOMEM;
    return MB_OK;
}

// Solve J delta = -R at the current c->u (FP64 residual in c->r) into c->du.
static int linear_solve(mb_cell* c, double dt, double rtol, int* its, double* relres, bool pc_setup = true) {
    int64_t n = c->n;
    cudaStream_t s = c->stream;
    k_convert<double, float><<<nblk(n), 256, 0, s>>>(c->u, c->u32, n), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("u32");
    int rc = set_dt(c, dt, s);
    if (rc) return rc;
    rc = c->opt.precision == MB_PREC_MIXED ? launch_lin_setup<float>(c, c->u32, c->gate, s)
                                           : launch_lin_setup<double>(c, c->u, c->gate, s);
    if (rc) return rc;
    if (pc_setup) {
        if ((rc = precond_setup(c, c->u32, c->gate, dt))) return rc;
        if ((rc = precond_setup_fine(c))) return rc;
    }
    if (!c->kd && (rc = krylov_create(c, &c->kd))) return rc;
    Krylov* K = c->kd;
    k_scale_rhs<<<nblk(n), 256, 0, s>>>(c->D, c->vcode, c->r, inv_scales(c, 1, dt), c->rowinv, K->b), ::mb::count_launch(c);
    OpCtx o{c->u32, c->gate, dt};
    rc = fgmres(c, K, o, rtol, c->opt.krylov_maxit, its, relres);
    if (!rc) rc = precond_check(c);
    if (rc) return rc;
    k_unscale<<<nblk(n), 256, 0, s>>>(c->P, c->D, c->vcode, K->x, c->du), ::mb::count_launch(c);
    MB_CUDA_LAUNCH("linear_solve");
    return MB_OK;
}

void krylov_destroy(mb_cell* c) {
    delete c->kd;
    c->kd = nullptr;
}

static constexpr double DELTA_MAX = 0.25;

// Newton with frozen gates for the step from c->u_old; c->u holds the start
// (from_old: u_old) and the result.
static int newton(mb_cell* c, double dt, double I_app, bool from_old, int* its_out, int* kits, double* rnorm_out,
                  bool* ok) {
    int64_t n = c->n;
    cudaStream_t s = c->stream;
    if (from_old) MB_CUDA(cudaMemcpyAsync(c->u, c->u_old, 8 * n, cudaMemcpyDeviceToDevice, s));
    *ok = false;
    double rn_prev = 0.0, eta_prev = 0.0;
    int base_its = 0, last_its = 0;   // Krylov iterations after the last preconditioner rebuild, and of the last solve
    double drift = 0.0;               // sum of the damped updates' scaled sizes since that rebuild
    double dn_prev = 0.0;             // scaled size of the previous update if it was a full step (else 0)
    for (int it = 1; it <= c->opt.newton_maxit; ++it) {
        int rc = launch_residual_split(c, c->u, c->u_old, c->gate, dt, I_app, c->r, s);
        if (rc) return rc;
        double rn;
        if ((rc = scaled_maxnorm(c, c->r, 1, dt, &rn))) return rc;
        *rnorm_out = rn;
        if (!(rn < 1e200)) { *its_out = it; return MB_OK; }
        // forcing term of the linear solve: fixed krylov_rtol, or (krylov_forcing
        // = 1) Eisenstat and Walker's choice 2, eta = 0.9 (|R_k| / |R_k-1|)^2
        // safeguarded by 0.9 eta_prev^2 when that exceeds 0.1, within
        // [krylov_rtol, 0.1] (0.1 at the first iteration)
        double eta = c->opt.krylov_rtol;
        if (c->opt.krylov_forcing) {
            if (it == 1) {
                eta = 0.1;
            } else {
                eta = 0.9 * (rn / rn_prev) * (rn / rn_prev);
                const double sg = 0.9 * eta_prev * eta_prev;
                if (sg > 0.1) eta = fmax(eta, sg);
            }
            eta = fmin(0.1, fmax(eta, c->opt.krylov_rtol));
        }
        rn_prev = rn;
        eta_prev = eta;
        int ki = 0;
        double rr = 0;
        // the preconditioner: rebuilt every iteration, or
        // (pc_lag) at the first, once the iterate has moved more than
        // pc_lag_drift since the previous rebuild, and whenever the last solve
        // needed clearly more iterations than the first after that rebuild
        bool setup = !c->opt.pc_lag || it == 1 || drift > c->opt.pc_lag_drift || last_its > 1.5 * base_its + 2;
        rc = linear_solve(c, dt, eta, &ki, &rr, setup);
        if (!setup && (rc == MB_ENOCONV || (rc == MB_OK && !(rr <= eta)))) {
            // the lagged preconditioner left the solve short of its tolerance:
            // rebuild it at the current iterate and solve again
            if (debug_level() > 0)
                fprintf(stderr, "[mb] newton it %d lagged solve missed its tolerance (krylov %d relres %.2e)\n", it,
                        ki, rr);
            *kits += ki;
            setup = true;
            rc = linear_solve(c, dt, eta, &ki, &rr, true);
        }
        if (rc == MB_ENOCONV) { *its_out = it; return MB_OK; }
        if (rc) return rc;
        if (setup) {
            base_its = ki;
            drift = 0.0;
        }
        last_its = ki;
        *kits += ki;
        // the step length caps the update of the voxel unknowns (c, phi: the
        // arguments of the exponentials) in their scales and of each plated
        // inventory relative to max(n_c, |n|): a stripping layer of many
        // critical thicknesses may change by a quarter of itself per iteration,
        // a thin one by a quarter of n_c (so that it does not overshoot into
        // n < 0, where f_pre switches off); convergence is tested on every
        // unknown in the fixed scales
        double dn, dv;
        if ((rc = scaled_maxnorm(c, c->du, 0, dt, &dn, &dv, c->u))) return rc;
        if (!(dn < 1e200)) { *its_out = it; return MB_OK; }
        double lam = dv <= DELTA_MAX ? 1.0 : DELTA_MAX / dv;
        drift += lam * dv;
        if (debug_level() > 0)
            fprintf(stderr, "[mb] newton it %d |R|_s %.3e |d|_s %.3e |d|_v %.3e lam %.3f krylov %d relres %.2e%s\n",
                    it, rn, dn, dv, lam, ki, rr, setup ? " rebuilt" : "");
        k_axpy_d<<<nblk(n), 256, 0, s>>>(lam, c->du, c->u, n), ::mb::count_launch(c);
        MB_CUDA_LAUNCH("newton update");
        if (c->snap_u) {   // record the Newton stage (reduced-model snapshots)
            c->snap_u->emplace_back(n);
            c->snap_g->emplace_back(c->D.F);
            MB_CUDA(cudaMemcpyAsync(c->snap_u->back().data(), c->u, 8 * n, cudaMemcpyDeviceToHost, s));
            if (c->D.F) MB_CUDA(cudaMemcpyAsync(c->snap_g->back().data(), c->gate, c->D.F, cudaMemcpyDeviceToHost, s));
            MB_CUDA(cudaStreamSynchronize(s));
        }
        // converged: the update is below the tolerance or, with newton_rate_test,
        // the error left after it is: estimated from the contraction of two full
        // steps (rho = |d_k| / |d_k-1|, remaining error ~ rho / (1 - rho) |d_k|)
        // plus the linear solve's own relative residual times |d_k|; a small
        // update only means convergence if the linear solve made progress
        bool small = lam * dn <= c->opt.newton_tol;
        if (!small && c->opt.newton_rate_test && lam == 1.0 && dn_prev > 0.0) {
            const double rho = dn / dn_prev;
            small = rho < 0.5 && (rho / (1.0 - rho) + rr) * dn <= c->opt.newton_tol;
        }
        dn_prev = lam == 1.0 ? dn : 0.0;
        if (small && rr <= fmax(0.5, eta)) {
            *its_out = it;
            *ok = true;
            return MB_OK;
        }
    }
    *its_out = c->opt.newton_maxit;
    return MB_OK;
}

// One step of size dt from c->u_old with the active-set passes; result in c->u.
static int try_step(mb_cell* c, double dt, double I_app, mb_step_info* info, bool* ok) {
    cudaStream_t s = c->stream;
    int64_t N = c->D.N, F = c->D.F;
    int rc = launch_gate(c, c->u_old, c->u_old + 2 * N, c->gate, s);
    if (rc) return rc;
    *ok = false;
    for (int pass = 1; pass <= c->opt.max_passes; ++pass) {
        int its = 0;
        double rn = 0;
        bool nok = false;
        // passes after the first start from the previous pass's converged state
        // when pass_start = 1 (the solution under the new gates differs from it
        // only near the flipped faces)
        const bool from_old = pass == 1 || c->opt.pass_start == 0;
        rc = newton(c, dt, I_app, from_old, &its, &info->krylov_its, &rn, &nok);
        if (rc) return rc;
        info->newton_its += its;
        info->passes = pass;
        info->res_norm = rn;
        if (!nok) return MB_OK;
        if (F == 0) { *ok = true; return MB_OK; }
        rc = launch_gate(c, c->u, c->u_old + 2 * N, c->gate2, s);
        if (rc) return rc;
        int64_t flips = 0;
        if ((rc = count_diff_u8(c, c->gate, c->gate2, F, &flips))) return rc;
        if (flips == 0) { *ok = true; return MB_OK; }
        if (pass == c->opt.max_passes) {
            // accepted with the last pass's gates; the faces that still flip are reported
            info->unresolved_flips += (int)flips;
            *ok = true;
            return MB_OK;
        }
        info->flips += (int)flips;
        MB_CUDA(cudaMemcpyAsync(c->gate, c->gate2, F, cudaMemcpyDeviceToDevice, s));
    }
    return MB_OK;
}

int newton_step(mb_cell* c, double dt, double I_app, mb_step_info* info) {
    memset(info, 0, sizeof(*info));
    int64_t n = c->n;
    cudaStream_t s = c->stream;
    MB_CUDA(cudaMemcpyAsync(c->u_pass, c->u, 8 * n, cudaMemcpyDeviceToDevice, s));
    // try the full step; on failure halve dt and take 2^h sub-steps
    for (int h = 0; h <= c->opt.max_halvings; ++h) {
        int nsub = 1 << h;
        double dts = dt / nsub;
        bool all_ok = true;
        info->unresolved_flips = 0;   // counts the sub-steps of the accepted attempt only
        MB_CUDA(cudaMemcpyAsync(c->u, c->u_pass, 8 * n, cudaMemcpyDeviceToDevice, s));
        for (int k = 0; k < nsub; ++k) {
            MB_CUDA(cudaMemcpyAsync(c->u_old, c->u, 8 * n, cudaMemcpyDeviceToDevice, s));
            bool ok = false;
            int rc = try_step(c, dts, I_app, info, &ok);
            if (rc) return rc;
            if (!ok) { all_ok = false; break; }
        }
        if (all_ok) {
            info->halvings = h;
            info->dt_used = dts;
            return functionals(c, c->u, info);
        }
    }
    MB_CUDA(cudaMemcpyAsync(c->u, c->u_pass, 8 * n, cudaMemcpyDeviceToDevice, s));
    MB_CUDA(cudaStreamSynchronize(s));
    set_error("Newton did not converge after all step halvings");
    return MB_ENOCONV;
}

// d = u_new - (u_start + r (u_start - u_hist)): the step's distance from the
// linear extrapolation of the two previous states (r = dt / dt_hist)
__global__ void k_lte_diff(const double* __restrict__ u_new, const double* __restrict__ u_start,
                           const double* __restrict__ u_hist, double r, double* __restrict__ d, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = u_new[i] - (u_start[i] + r * (u_start[i] - u_hist[i]));
}

// One accepted adaptive step (see mb_step_adaptive): local error e =
// dt/(2 dt + dt_hist) |u_new - u_pred|_s, retries with dt * clamp(0.9
// sqrt(tol/e), 0.2, 2) while e > tol.
int adaptive_step(mb_cell* c, double dt_try, double I_app, const mb_adapt_opts* o, mb_adapt_info* ai,
                  mb_step_info* info) {
    const int64_t n = c->n;
    cudaStream_t s = c->stream;
    if (!c->u_hist) {
        c->u_hist = (double*)cell_alloc(c, 8 * (size_t)n);
        c->u_save = (double*)cell_alloc(c, 8 * (size_t)n);
        if (!c->u_hist || !c->u_save) { set_error("mb_step_adaptive: device memory"); return MB_ENOMEM; }
    }
    memset(ai, 0, sizeof(*ai));
    mb_step_info sum;
    memset(&sum, 0, sizeof(sum));
    double dt = fmin(fmax(dt_try, o->dt_min), o->dt_max);
    MB_CUDA(cudaMemcpyAsync(c->u_save, c->u, 8 * n, cudaMemcpyDeviceToDevice, s));
    for (int rejects = 0;; ++rejects) {
        mb_step_info one;
        int rc = newton_step(c, dt, I_app, &one);
        sum.newton_its += one.newton_its;
        sum.krylov_its += one.krylov_its;
        sum.flips += one.flips;
        if (rc) {
            *info = sum;
            return rc;
        }
        double e = 0.0, fac = 1.0;
        const bool hist = c->has_hist;
        if (hist) {
            k_lte_diff<<<nblk(n), 256, 0, s>>>(c->u, c->u_save, c->u_hist, dt / c->dt_hist, c->du, n),
                ::mb::count_launch(c);
            MB_CUDA_LAUNCH("lte_diff");
            if ((rc = scaled_maxnorm(c, c->du, 0, dt, &e))) return rc;
            e *= dt / (2.0 * dt + c->dt_hist);
            fac = e == 0.0 ? 2.0 : fmin(2.0, fmax(0.2, 0.9 * sqrt(o->tol / e)));
        }
        if (!hist || e <= o->tol || dt <= o->dt_min || rejects >= o->max_rejects) {
            // accept: the start of this step becomes the history
            std::swap(c->u_hist, c->u_save);
            c->dt_hist = dt;
            c->has_hist = true;
            ai->dt_used = dt;
            ai->dt_next = hist ? fmin(fmax(dt * fac, o->dt_min), o->dt_max) : dt;
            ai->err = e;
            ai->rejects = rejects;
            const int nits = sum.newton_its, kits = sum.krylov_its, flips = sum.flips;
            *info = one;
            info->newton_its = nits;
            info->krylov_its = kits;
            info->flips = flips;
            return MB_OK;
        }
        // reject: back to the start, smaller step
        MB_CUDA(cudaMemcpyAsync(c->u, c->u_save, 8 * n, cudaMemcpyDeviceToDevice, s));
        dt = fmax(dt * fac, o->dt_min);
    }
}

}  // namespace mb
