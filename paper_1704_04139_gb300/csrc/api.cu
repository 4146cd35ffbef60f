// api.cu -- extern "C" entry points of libmb (declared in include/mb.h).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <string>

#include "mb_internal.h"

namespace mb {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return MB_ECUDA;
}

void* cell_alloc(mb_cell* c, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc failed (" + std::to_string(bytes) + " bytes)");
        return nullptr;
    }
    c->owned.push_back(DBuf{p, bytes});
    c->device_bytes += (int64_t)bytes;
    return p;
}

static void fill_devparams(const mb_params& p, double h, DevParams& P) {
    memset(&P, 0, sizeof(P));
    P.h = h;
    P.A = h * h;
    P.V = h * h * h;
    double RT = p.R * p.T;
    P.invF = 1.0 / p.F;
    P.f2 = p.F / (2.0 * RT);
    P.E_gD = P.A * p.E_D / h;
    P.E_gk = P.A * p.E_kappa / h;
    P.E_gm = P.A * 2.0 * p.E_kappa * (p.E_tplus - 1.0) * (RT / p.F) * p.E_tdf / h;
    P.E_tF = p.E_tplus / p.F;
    for (int i = 0; i < 6; ++i) { P.cmin[i] = 0.0; P.cref[i] = 1.0; }
    P.cmin[PE] = p.clamp_rel * p.E_c0;
    P.cmin[PG] = p.clamp_rel * p.G_cmax;
    P.cmin[PK] = p.clamp_rel * p.K_cmax;
    P.cref[PE] = p.E_c0;
    P.cref[PG] = p.G_cmax;
    P.cref[PK] = p.K_cmax;
    P.gD[PG] = P.A * p.G_D / h;
    P.gD[PK] = P.A * p.K_D / h;
    double sig[6] = {0.0, p.G_sigma, p.K_sigma, p.L_sigma, p.CN_sigma, p.CP_sigma};
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 6; ++b)
            P.gsig[a][b] = (sig[a] > 0 && sig[b] > 0) ? P.A * (2.0 * sig[a] * sig[b] / (sig[a] + sig[b])) / h : 0.0;
    P.i00[PG] = p.G_i00;
    P.i00[PK] = p.K_i00;
    P.i00[PL] = p.L_i00;
    P.icmax[PG] = 1.0 / p.G_cmax;
    P.icmax[PK] = 1.0 / p.K_cmax;
    for (int i = 0; i < 7; ++i) { P.ocpG[i] = p.G_ocp[i]; P.ocpK[i] = p.K_ocp[i]; }
    P.g_dir = 2.0 * P.A * p.CN_sigma / h;
    P.Pl_i00 = p.Pl_i00;
    double nc = p.Pl_layer_m / p.Pl_Vm_Li;
    P.nc4 = nc * nc * nc * nc;
    P.nc = nc;
}

cudaEvent_t Prof::get() {
    if (used == pool.size()) {
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        pool.push_back(e);
    }
    return pool[used++];
}

static void free_cell(mb_cell* c) {
    if (!c) return;
    for (auto e : c->prof.pool) cudaEventDestroy(e);
    precond_destroy(c);
    krylov_destroy(c);
    for (auto& b : c->owned) cudaFree(b.p);
    if (c->h_red) cudaFreeHost(c->h_red);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // namespace mb

using namespace mb;

extern "C" {

const char* mb_last_error(void) { return g_err.c_str(); }

void mb_opts_default(mb_solver_opts* o) {
    if (!o) return;
    o->precision = MB_PREC_FP64;
    o->newton_tol = 1e-12;
    o->newton_maxit = 30;
    o->gmres_m = 30;
    o->krylov_maxit = 600;
    o->krylov_rtol = 1e-6;
    o->max_passes = 3;
    o->max_halvings = 6;
    o->mg_coarse_cells = 32;
    o->mg_smooth = 2;
    o->mg_kcycle = 5;
    o->mg_coarse_pre = 2;
    o->mg_coarse_post = 2;
    o->mg_bf16 = 1;
    o->mg_stream = 3;
    o->pass_start = 1;
    o->mg_kcycle_reorth = 1;
    o->krylov_forcing = 1;
    o->mg_tail = 0;
    o->pc_lag = 1;
    o->pc_lag_drift = 0.05;
    o->mg_pdl = 0;
    o->newton_rate_test = 1;
}

static int check_opts(const mb_solver_opts* o) {
    if (o->precision != MB_PREC_FP64 && o->precision != MB_PREC_MIXED) return MB_EINVAL;
    // gmres_m + 1 dot products must fit the 64-slot reduction buffers
    if (o->gmres_m < 1 || o->gmres_m > 63 || o->newton_maxit < 1 || o->krylov_maxit < 1 ||
        o->max_passes < 1 || o->max_halvings < 0 || o->max_halvings > 20 || !(o->newton_tol > 0) ||
        !(o->krylov_rtol > 0) || o->mg_kcycle < 1 || o->mg_kcycle > 16 || o->mg_smooth < 1 || o->mg_smooth > 8 ||
        (o->mg_bf16 != 0 && o->mg_bf16 != 1) || o->mg_coarse_pre < 1 || o->mg_coarse_pre > 4 ||
        o->mg_coarse_post < 1 || o->mg_coarse_post > 4 || o->mg_stream < 0 || o->mg_stream > 3 ||
        (o->pass_start != 0 && o->pass_start != 1) || o->mg_tail < 0 || o->mg_tail > 16 || (o->pc_lag != 0 && o->pc_lag != 1) || !(o->pc_lag_drift >= 0) || (o->mg_pdl != 0 && o->mg_pdl != 1) || (o->newton_rate_test != 0 && o->newton_rate_test != 1) ||
        (o->krylov_forcing != 0 && o->krylov_forcing != 1) ||
        (o->mg_kcycle_reorth != 0 && o->mg_kcycle_reorth != 1))
        return MB_EINVAL;
    return MB_OK;
}

int mb_cell_create(const uint8_t* labels, int nt, int ny, int nz, double h, const mb_params* p,
                   const mb_solver_opts* o, mb_cell** out) {
    if (!labels || !p || !out || nt < 1 || ny < 1 || nz < 1 || !(h > 0)) {
        set_error("mb_cell_create: invalid argument");
        return MB_EINVAL;
    }
    *out = nullptr;
    mb_solver_opts opt;
    mb_opts_default(&opt);
    if (o) opt = *o;
    if (check_opts(&opt)) { set_error("mb_cell_create: invalid solver options"); return MB_EINVAL; }
    if (nt > 65535) { set_error("mb_cell_create: nt must be <= 65535"); return MB_EINVAL; }
    int64_t N = (int64_t)nt * ny * nz;
    if (N >= (int64_t)1 << 31) { set_error("mb_cell_create: grid too large for 32-bit voxel indices"); return MB_EINVAL; }
    mb_cell* c = new mb_cell();
    c->prm = *p;
    c->opt = opt;
    cudaGetDevice(&c->device);
    c->D.nt = nt; c->D.ny = ny; c->D.nz = nz; c->D.N = N; c->D.syz = (int64_t)ny * nz; c->D.F = 0;
    fill_devparams(*p, h, c->P);
    par_convert(c->P, c->Pf);
    for (int64_t i = 0; i < N; ++i) {
        if (labels[i] > 5) { set_error("mb_cell_create: labels must be in 0..5"); delete c; return MB_EINVAL; }
        c->count[labels[i]]++;
    }
    int rc = MB_OK;
    uint8_t* d_lab = nullptr;
    do {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "cudaStreamCreate"); break;
        }
        if (cudaMallocHost(&c->h_red, 64 * 8) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "cudaMallocHost"); break; }
        if (cudaMalloc(&d_lab, N) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "cudaMalloc"); break; }
        if (cudaMemcpyAsync(d_lab, labels, N, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "copy labels"); break;
        }
        if ((rc = launch_classify(c, d_lab))) break;
        int64_t n = c->n;
        size_t F = c->D.F ? c->D.F : 1;
        c->u = (double*)cell_alloc(c, 8 * n);
        c->u_old = (double*)cell_alloc(c, 8 * n);
        c->u_pass = (double*)cell_alloc(c, 8 * n);
        c->r = (double*)cell_alloc(c, 8 * n);
        c->du = (double*)cell_alloc(c, 8 * n);
        c->u32 = (float*)cell_alloc(c, 4 * n);
        c->gate = (uint8_t*)cell_alloc(c, F);
        c->gate2 = (uint8_t*)cell_alloc(c, F);
        c->red = (double*)cell_alloc(c, 8 * (size_t)RED_BLOCKS * 64);
        c->red_out = (double*)cell_alloc(c, 8 * 64);
        c->icoef = (float*)cell_alloc(c, 4 * (size_t)NCOEF * (c->D.NI ? c->D.NI : 1));
        c->d_dtinv = (float*)cell_alloc(c, 256);
        c->icur = (double*)cell_alloc(c, 16 * (size_t)(c->D.NI ? c->D.NI : 1));
        if (!c->u || !c->u_old || !c->u_pass || !c->r || !c->du || !c->u32 || !c->gate || !c->gate2 ||
            !c->red || !c->red_out || !c->icoef || !c->d_dtinv || !c->icur) { rc = MB_ENOMEM; break; }
        if ((rc = launch_init_state(c, c->u))) break;
        if ((rc = precond_create(c))) break;
        double nG = (double)c->count[PG];
        c->i_1c = p->F * c->P.V * p->G_cmax * (1.0 - p->G_x0) * nG / 3600.0 / ((double)ny * nz * c->P.A);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "create sync"); break; }
    } while (0);
    if (d_lab) cudaFree(d_lab);
    if (rc) { free_cell(c); return rc; }
    *out = c;
    return MB_OK;
}

int mb_cell_destroy(mb_cell* c) {
    if (!c) { set_error("mb_cell_destroy: invalid argument"); return MB_EINVAL; }
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_cell(c);
    return MB_OK;
}

int mb_cell_info_get(mb_cell* c, mb_cell_info* info) {
    if (!c || !info) { set_error("mb_cell_info_get: invalid argument"); return MB_EINVAL; }
    info->n_vox = c->D.N;
    info->n_faces = c->D.F;
    info->n_unknowns = c->n;
    info->nt = c->D.nt; info->ny = c->D.ny; info->nz = c->D.nz;
    info->h = c->P.h;
    info->i_1c = c->i_1c;
    for (int i = 0; i < 6; ++i) info->count[i] = c->count[i];
    info->device_bytes = c->device_bytes;
    info->n_iface = c->D.NI;
    return MB_OK;
}

int mb_cell_set_scales(mb_cell* c, double s_i0, double k_pl) {
    if (!c || !(s_i0 >= 0) || !(k_pl >= 0)) { set_error("mb_cell_set_scales: invalid argument"); return MB_EINVAL; }
    c->s_i0 = s_i0;
    c->k_pl = k_pl;
    return MB_OK;
}

int mb_cell_set_opts(mb_cell* c, const mb_solver_opts* o) {
    if (!c || !o || check_opts(o)) { set_error("mb_cell_set_opts: invalid options"); return MB_EINVAL; }
    bool remake = o->gmres_m != c->opt.gmres_m;
    c->opt = *o;
    if (remake) {
        // Krylov workspaces are re-created lazily with the new restart length
        // (their old buffers stay owned by the cell until it is destroyed)
        krylov_destroy(c);
    }
    return MB_OK;
}

int mb_plating_faces(mb_cell* c, int32_t* g, int32_t* e, int32_t* dir) {
    if (!c) { set_error("mb_plating_faces: invalid argument"); return MB_EINVAL; }
    int64_t F = c->D.F;
    if (F == 0) return MB_OK;
    if (g) MB_CUDA(cudaMemcpy(g, c->pf_g, 4 * F, cudaMemcpyDeviceToHost));
    if (e) MB_CUDA(cudaMemcpy(e, c->pf_e, 4 * F, cudaMemcpyDeviceToHost));
    if (dir) {
        std::vector<int8_t> tmp(F);
        MB_CUDA(cudaMemcpy(tmp.data(), c->pf_dir, F, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < F; ++i) dir[i] = tmp[i];
    }
    return MB_OK;
}

int mb_state_get(mb_cell* c, double* u) {
    if (!c || !u) { set_error("mb_state_get: invalid argument"); return MB_EINVAL; }
    MB_CUDA(cudaMemcpyAsync(u, c->u, 8 * c->n, cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(cudaStreamSynchronize(c->stream));
    return MB_OK;
}

int mb_state_set(mb_cell* c, const double* u) {
    if (!c || !u) { set_error("mb_state_set: invalid argument"); return MB_EINVAL; }
    MB_CUDA(cudaMemcpyAsync(c->u, u, 8 * c->n, cudaMemcpyHostToDevice, c->stream));
    MB_CUDA(cudaStreamSynchronize(c->stream));
    c->has_hist = false;
    return MB_OK;
}

int mb_step(mb_cell* c, double dt, double I_app, mb_step_info* info) {
    if (!c || !(dt > 0) || !(fabs(I_app) < 1e300)) { set_error("mb_step: invalid argument"); return MB_EINVAL; }
    mb_step_info tmp;
    c->has_hist = false;   // a fixed step ends the adaptive history
    return newton_step(c, dt, I_app, info ? info : &tmp);
}

int mb_step_adaptive(mb_cell* c, double dt_try, double I_app, const mb_adapt_opts* o, mb_adapt_info* ai,
                     mb_step_info* info) {
    if (!c || !o || !(dt_try > 0) || !(fabs(I_app) < 1e300) || !(o->tol > 0) || !(o->dt_min > 0) ||
        !(o->dt_max >= o->dt_min) || o->max_rejects < 0) {
        set_error("mb_step_adaptive: invalid argument");
        return MB_EINVAL;
    }
    mb_step_info tmp;
    mb_adapt_info atmp;
    return adaptive_step(c, dt_try, I_app, o, ai ? ai : &atmp, info ? info : &tmp);
}

int mb_adapt_reset(mb_cell* c) {
    if (!c) { set_error("mb_adapt_reset: invalid argument"); return MB_EINVAL; }
    c->has_hist = false;
    return MB_OK;
}

int mb_residual_dev(mb_cell* c, const double* u, const double* u_old, const uint8_t* gate, double dt,
                    double I_app, double* r, void* stream) {
    if (!c || !u || !u_old || !r || !(dt > 0)) { set_error("mb_residual_dev: invalid argument"); return MB_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const uint8_t* g = gate;
    if (!g) {
        int rc = launch_gate(c, u_old, u_old + 2 * c->D.N, c->gate2, s);
        if (rc) return rc;
        g = c->gate2;
    }
    int rc = launch_residual<double>(c, u, u_old, g, dt, I_app, r, s);
    if (rc) return rc;
    MB_CUDA(cudaStreamSynchronize(s));
    return MB_OK;
}

int mb_residual(mb_cell* c, const double* u, const double* u_old, const uint8_t* gate, double dt,
                double I_app, double* r) {
    if (!c || !u || !u_old || !r || !(dt > 0)) { set_error("mb_residual: invalid argument"); return MB_EINVAL; }
    int64_t n = c->n, F = c->D.F;
    cudaStream_t s = c->stream;
    MB_CUDA(cudaMemcpyAsync(c->du, u, 8 * n, cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemcpyAsync(c->u_pass, u_old, 8 * n, cudaMemcpyHostToDevice, s));
    const uint8_t* g = nullptr;
    if (gate && F) {
        MB_CUDA(cudaMemcpyAsync(c->gate2, gate, F, cudaMemcpyHostToDevice, s));
        g = c->gate2;
    }
    int rc = mb_residual_dev(c, c->du, c->u_pass, g ? g : (F ? nullptr : c->gate2), dt, I_app, c->r, s);
    if (rc) return rc;
    MB_CUDA(cudaMemcpyAsync(r, c->r, 8 * n, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    return MB_OK;
}

int mb_jvp_dev(mb_cell* c, const double* u, const uint8_t* gate, double dt, const double* v, double* jv,
               void* stream) {
    if (!c || !u || !v || !jv || !(dt > 0)) { set_error("mb_jvp_dev: invalid argument"); return MB_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const uint8_t* g = gate;
    if (!g) {
        int rc = launch_gate(c, u, u + 2 * c->D.N, c->gate2, s);
        if (rc) return rc;
        g = c->gate2;
    }
    int rc = launch_jvp<double, double>(c, u, g, dt, v, jv, s);
    if (rc) return rc;
    MB_CUDA(cudaStreamSynchronize(s));
    return MB_OK;
}

int mb_jvp(mb_cell* c, const double* u, const uint8_t* gate, double dt, const double* v, double* jv) {
    if (!c || !u || !v || !jv || !(dt > 0)) { set_error("mb_jvp: invalid argument"); return MB_EINVAL; }
    int64_t n = c->n, F = c->D.F;
    cudaStream_t s = c->stream;
    MB_CUDA(cudaMemcpyAsync(c->du, u, 8 * n, cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemcpyAsync(c->u_pass, v, 8 * n, cudaMemcpyHostToDevice, s));
    const uint8_t* g = nullptr;
    if (gate && F) {
        MB_CUDA(cudaMemcpyAsync(c->gate2, gate, F, cudaMemcpyHostToDevice, s));
        g = c->gate2;
    }
    int rc = mb_jvp_dev(c, c->du, g ? g : (F ? nullptr : c->gate2), dt, c->u_pass, c->r, s);
    if (rc) return rc;
    MB_CUDA(cudaMemcpyAsync(jv, c->r, 8 * n, cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    return MB_OK;
}

int mb_jvp_f32_dev(mb_cell* c, const float* u, const uint8_t* gate, double dt, const float* v, float* jv,
                   void* stream) {
    if (!c || !u || !v || !jv || !(dt > 0) || (!gate && c->D.F)) {
        set_error("mb_jvp_f32_dev: invalid argument (gate is required when the cell has plating faces)");
        return MB_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_jvp<float, float>(c, u, gate ? gate : c->gate2, dt, v, jv, s);
    if (rc) return rc;
    MB_CUDA(cudaStreamSynchronize(s));
    return MB_OK;
}

}  // extern "C"

extern "C" {

int mb_prof_enable(mb_cell* c, int on) {
    if (!c) { set_error("mb_prof_enable: invalid argument"); return MB_EINVAL; }
    cudaStreamSynchronize(c->stream);
    precond_harvest(c);
    c->prof.enabled = on != 0;
    for (auto& r : c->prof.rec) r.clear();
    for (int k = 0; k < PROF_NKERNELS; ++k) { c->prof.acc_ms[k] = 0.0; c->prof.acc_n[k] = 0; }
    c->prof.used = 0;
    return MB_OK;
}

int mb_prof_read(mb_cell* c, int kind, int64_t* count, double* total_ms) {
    if (!c || kind < 0 || kind >= PROF_NKERNELS || !count || !total_ms) {
        set_error("mb_prof_read: invalid argument");
        return MB_EINVAL;
    }
    MB_CUDA(cudaStreamSynchronize(c->stream));
    precond_harvest(c);
    double tot = c->prof.acc_ms[kind];
    for (auto& pr : c->prof.rec[kind]) {
        float ms = 0.f;
        MB_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
        tot += ms;
    }
    *count = (int64_t)c->prof.rec[kind].size() + c->prof.acc_n[kind];
    *total_ms = tot;
    return MB_OK;
}

int mb_prof_reset(mb_cell* c) {
    if (!c) return MB_EINVAL;
    cudaStreamSynchronize(c->stream);
    precond_harvest(c);
    for (auto& r : c->prof.rec) r.clear();
    for (int k = 0; k < PROF_NKERNELS; ++k) { c->prof.acc_ms[k] = 0.0; c->prof.acc_n[k] = 0; }
    c->prof.used = 0;
    return MB_OK;
}

int mb_cell_stream(mb_cell* c, void** stream) {
    if (!c || !stream) { set_error("mb_cell_stream: invalid argument"); return MB_EINVAL; }
    *stream = (void*)c->stream;
    return MB_OK;
}

int mb_launch_count(mb_cell* c, int64_t* count) {
    if (!c || !count) { set_error("mb_launch_count: invalid argument"); return MB_EINVAL; }
    *count = c->launches;
    return MB_OK;
}

}  // extern "C"
