// mb_model.cuh -- device-side model of the voxel finite-volume operator.
//
// Per-face fluxes of the cell-centred finite volume scheme (Sec. 2.4) for the
// transport equations of Sec. 2.2 (Eqs. cgr, phigr, cel, phiel), the
// interface conditions of Eq. (interfaceCond) with the kinetics of
// Eqs. (ise_gr), (ise_li) and the plating/stripping kinetics of Eq. (iplel)
// with the regulariser f_pre of Sec. 2.3.  Everything is written from the
// point of view of one voxel v and one neighbour w; the face's contribution
// to v's rows is returned.  T is double (outer Newton residual, FP64
// linearisation) or float (Jacobian coefficients of the preconditioner and
// of the mixed-precision Krylov operator).
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

namespace mb {

enum Phase : int { PE = 0, PG = 1, PK = 2, PL = 3, PCN = 4, PCP = 5 };

// per-voxel code: bits 0-2 phase, bits 3-8 mask of electrolyte neighbours of a
// solid voxel with interface kinetics (G, K, L; bit d = direction d), bits
// 9-31 index of its first interface face (for G: its first plating face)
constexpr int VC_FBASE_SHIFT = 9;
constexpr uint32_t VC_MAX_FACES = (1u << 23);
__host__ __device__ inline int vc_phase(uint32_t c) { return int(c & 7u); }
__host__ __device__ inline uint32_t vc_emask(uint32_t c) { return (c >> 3) & 63u; }
__host__ __device__ inline uint32_t vc_fbase(uint32_t c) { return c >> VC_FBASE_SHIFT; }
__device__ inline int opp_dir(int d) { return d ^ 1; }

struct Dims {
    int nt, ny, nz;
    int64_t N;      // voxels
    int64_t F;      // plating faces (graphite-electrolyte)
    int64_t NI;     // interface faces: plating faces, then cathode/foil-electrolyte faces
    int64_t syz;    // ny*nz
};

// Constants of the model with the voxel geometry folded in (A = h^2), in
// the arithmetic type T of the kernels that read them: the FP32 kernels get
// an FP32 copy so that no parameter is converted from FP64 on the device.
// Every member has type T (par_convert relies on that).
template <class T>
struct ParT {
    T h, A, V;
    T invF, f2;                    // 1/F, F/(2RT)
    T E_gD;                        // A D_E / h
    T E_gk;                        // A kappa / h
    T E_gm;                        // A 2 kappa (t+ - 1) (RT/F) TDF / h  (divided by c_a + c_b)
    T E_tF;                        // t+ / F
    T cmin[6];                     // concentration clamp per phase
    T cref[6];                     // concentration scale per phase (1 where no c)
    T gD[6];                       // A D_s / h for G, K
    T gsig[6][6];                  // A sigma_face / h for conductor pairs (harmonic mean)
    T i00[6];                      // BV prefactor per solid phase (G, K: i00; L: i00_L)
    T icmax[6];
    T ocpG[7], ocpK[7];
    T g_dir;                       // 2 A sigma_CN / h  (Dirichlet half-voxel ghost)
    T Pl_i00, nc4, nc;             // plating prefactor, n_c^4, n_c
};
using DevParams = ParT<double>;
using DevParamsF = ParT<float>;

// member-wise conversion (both structs are plain arrays of their type)
template <class A, class B>
inline void par_convert(const ParT<A>& a, ParT<B>& b) {
    static_assert(sizeof(ParT<A>) / sizeof(A) == sizeof(ParT<B>) / sizeof(B), "ParT layout");
    const A* src = reinterpret_cast<const A*>(&a);
    B* dst = reinterpret_cast<B*>(&b);
    for (size_t i = 0; i < sizeof(ParT<A>) / sizeof(A); ++i) dst[i] = B(src[i]);
}

__host__ __device__ inline bool is_conductor(int p) { return p != PE; }
__host__ __device__ inline bool has_c(int p) { return p == PE || p == PG || p == PK; }

template <class T> __device__ inline T tmax(T a, T b) { return a > b ? a : b; }

// 1/S in FP64 on the FMA pipe: the FP32 reciprocal refined by two
// Newton-Raphson steps x <- x + x (1 - S x), each of which squares the
// relative error (2^-24 -> 2^-48 -> below the FP64 rounding of the last FMA),
// so the result is within ~1 ulp of 1/S.  Outside the FP32 exponent range
// the plain division.
__device__ inline double rcp_nr(double S) {
    const double a = fabs(S);
    if (!(a > 1e-30 && a < 1e30)) return 1.0 / S;
    double x = (double)__frcp_rn((float)S);
    double e = fma(-S, x, 1.0);
    x = fma(x, e, x);
    e = fma(-S, x, 1.0);
    return fma(x, e, x);
}

template <class T>
__device__ inline T ocp_val(const T* a, T x) {
    return T(a[0]) + T(a[1]) * x + T(a[2]) * exp(-T(a[3]) * x) + T(a[4]) * tanh((x - T(a[5])) / T(a[6]));
}
template <class T>
__device__ inline T ocp_der(const T* a, T x) {   // dU0/dx
    T th = tanh((x - T(a[5])) / T(a[6]));
    return T(a[1]) - T(a[2]) * T(a[3]) * exp(-T(a[3]) * x) + T(a[4]) / T(a[6]) * (T(1) - th * th);
}

// Interface current density from solid s into electrolyte e (A/m^2):
// Butler-Volmer part ibv (Eq. ise_gr for G and K, Eq. ise_li for L) and the
// plating part ipl (Eq. iplel, graphite faces with an active gate).
template <class T>
__device__ inline void interface_current(const ParT<T>& P, int ls, T cs, T ps, T ce, T pe, T nf,
                                         bool gate, T s_i0, T k_pl, T& ibv, T& ipl) {
    const T f2 = T(P.f2);
    ipl = T(0);
    if (ls == PL) {
        ibv = T(2) * T(P.i00[PL]) * sinh(f2 * (ps - pe));
        return;
    }
    T csa = tmax(cs, T(P.cmin[ls]));
    T cea = tmax(ce, T(P.cmin[PE]));
    T x = csa * T(P.icmax[ls]);
    T U = ocp_val<T>(ls == PG ? P.ocpG : P.ocpK, x);
    T eta = ps - U - pe;
    ibv = T(2) * T(P.i00[ls]) * s_i0 * sqrt(csa * cea) * sinh(f2 * eta);
    if (ls == PG && gate) {
        T etap = ps - pe;
        T np = tmax(nf, T(0));
        T n4 = np * np * np * np;
        T fpre = n4 / (T(P.nc4) + n4);
        ipl = k_pl * T(P.Pl_i00) * sqrt(cea) * (fpre * exp(f2 * etap) - exp(-f2 * etap));
    }
}

// Contribution of face (v, w) to v's rows R_c(v), R_phi(v); for a graphite
// v next to electrolyte w also returns i_pl (for the face row R_n).
template <class T>
__device__ inline void face_residual(const ParT<T>& P, int lv, int lw, T cv, T pv, T cw, T pw,
                                     T nf, bool gate, T s_i0, T k_pl, T& rc, T& rp, T& ipl_out) {
    if (lv == PE && lw == PE) {
        T S = tmax(cv, T(P.cmin[PE])) + tmax(cw, T(P.cmin[PE]));
        T dc = cw - cv, dp = pw - pv;
        T j = -T(P.E_gk) * dp - T(P.E_gm) * dc / S;        // A * current density
        rc += -T(P.E_gD) * dc + T(P.E_tF) * j;
        rp += j;
    } else if (lv == lw && (lv == PG || lv == PK)) {
        rc += -T(P.gD[lv]) * (cw - cv);
        rp += -T(P.gsig[lv][lw]) * (pw - pv);
    } else if (is_conductor(lv) && is_conductor(lw)) {
        rp += -T(P.gsig[lv][lw]) * (pw - pv);
    } else if (lw == PE && (lv == PG || lv == PK || lv == PL)) {
        T ibv, ipl;
        interface_current<T>(P, lv, cv, pv, cw, pw, nf, gate, s_i0, k_pl, ibv, ipl);
        if (lv != PL) rc += T(P.A) * ibv * T(P.invF);
        rp += T(P.A) * (ibv + ipl);
        ipl_out = ipl;
    } else if (lv == PE && (lw == PG || lw == PK || lw == PL)) {
        T ibv, ipl;
        interface_current<T>(P, lw, cw, pw, cv, pv, nf, gate, s_i0, k_pl, ibv, ipl);
        rc -= T(P.A) * (ibv + ipl) * T(P.invF);
        rp -= T(P.A) * (ibv + ipl);
    }
}

// Partial derivatives of one face's contribution to v's rows with respect to
// x = (c_v, phi_v, c_w, phi_w, n_f):  c[k] = d R_c(v)/d x_k, p[k] = d R_phi(v)/d x_k,
// and for a graphite v next to electrolyte w, n[k] = d (i_pl/F)/d x_k (face row).
template <class T>
struct FaceJac {
    T c[5], p[5], n[5];
};

template <class T>
__device__ inline void interface_partials(const ParT<T>& P, int ls, T cs, T ps, T ce, T pe, T nf,
                                          bool gate, T s_i0, T k_pl,
                                          T& i_eta, T& i_cs, T& i_ce,
                                          T& ip_eta, T& ip_ce, T& ip_n) {
    const T f2 = T(P.f2);
    ip_eta = ip_ce = ip_n = T(0);
    if (ls == PL) {
        i_eta = T(2) * T(P.i00[PL]) * f2 * cosh(f2 * (ps - pe));
        i_cs = i_ce = T(0);
        return;
    }
    T ms = cs >= T(P.cmin[ls]) ? T(1) : T(0);
    T me = ce >= T(P.cmin[PE]) ? T(1) : T(0);
    T csa = tmax(cs, T(P.cmin[ls]));
    T cea = tmax(ce, T(P.cmin[PE]));
    const T* a = ls == PG ? P.ocpG : P.ocpK;
    T x = csa * T(P.icmax[ls]);
    T eta = ps - ocp_val<T>(a, x) - pe;
    T k0 = T(2) * T(P.i00[ls]) * s_i0;
    T q = sqrt(csa * cea);
    T sh = sinh(f2 * eta), ch = cosh(f2 * eta);
    i_eta = k0 * q * f2 * ch;
    i_cs = ms * (k0 * q / (T(2) * csa) * sh - i_eta * ocp_der<T>(a, x) * T(P.icmax[ls]));
    i_ce = me * k0 * q / (T(2) * cea) * sh;
    if (ls == PG && gate) {
        T etap = ps - pe;
        T ep = exp(f2 * etap), em = exp(-f2 * etap);
        T np = tmax(nf, T(0));
        T n2 = np * np, n4 = n2 * n2;
        T den = T(P.nc4) + n4;
        T fpre = n4 / den;
        T dfpre = nf > T(0) ? T(4) * n2 * np * T(P.nc4) / (den * den) : T(0);
        T k1 = k_pl * T(P.Pl_i00);
        T rce = sqrt(cea);
        ip_eta = k1 * rce * f2 * (fpre * ep + em);
        ip_ce = me * k1 / (T(2) * rce) * (fpre * ep - em);
        ip_n = k1 * rce * dfpre * ep;
    }
}

// interface-face entries of J from the six partials; solid_side: v is the
// solid voxel (x = (c_s, phi_s, c_e, phi_e, n)), else the electrolyte voxel
// (x = (c_e, phi_e, c_s, phi_s, n))
template <class T>
__device__ inline void face_jacobian_iface(const ParT<T>& P, bool solid_side, bool solid_has_c, T i_eta, T i_cs,
                                           T i_ce, T ip_eta, T ip_ce, T ip_n, FaceJac<T>& J) {
    T A = T(P.A), AF = T(P.A) * T(P.invF), iF = T(P.invF);
    if (solid_side) {
        if (solid_has_c) {
            J.c[0] = AF * i_cs; J.c[1] = AF * i_eta; J.c[2] = AF * i_ce; J.c[3] = -AF * i_eta;
        }
        J.p[0] = A * i_cs; J.p[1] = A * (i_eta + ip_eta); J.p[2] = A * (i_ce + ip_ce);
        J.p[3] = -A * (i_eta + ip_eta); J.p[4] = A * ip_n;
        J.n[1] = iF * ip_eta; J.n[2] = iF * ip_ce; J.n[3] = -iF * ip_eta; J.n[4] = iF * ip_n;
    } else {
        T te = i_eta + ip_eta;
        J.c[0] = -AF * (i_ce + ip_ce); J.c[1] = AF * te; J.c[2] = -AF * i_cs; J.c[3] = -AF * te;
        J.c[4] = -AF * ip_n;
        J.p[0] = -A * (i_ce + ip_ce); J.p[1] = A * te; J.p[2] = -A * i_cs; J.p[3] = -A * te;
        J.p[4] = -A * ip_n;
        // face row i_pl/F seen from the electrolyte side: x = (c_e, phi_e, c_g, phi_g, n)
        J.n[0] = iF * ip_ce; J.n[1] = -iF * ip_eta; J.n[3] = iF * ip_eta; J.n[4] = iF * ip_n;
    }
}

// the face types without interface kinetics; false for an interface face (J untouched then)
template <class T>
__device__ inline bool face_jacobian_bulk(const ParT<T>& P, int lv, int lw, T cv, T cw, FaceJac<T>& J) {
    if (lv == PE && lw == PE) {
        T cmin = T(P.cmin[PE]);
        T mv = cv >= cmin ? T(1) : T(0), mw = cw >= cmin ? T(1) : T(0);
        T S = tmax(cv, cmin) + tmax(cw, cmin);
        T iS = T(1) / S;
        T dc = cw - cv;
        T r = dc * iS * iS;
        T gm = T(P.E_gm), gk = T(P.E_gk), tF = T(P.E_tF), gD = T(P.E_gD);
        T jcv = gm * (iS + r * mv);       // d j / d c_v
        T jcw = -gm * (iS - r * mw);      // d j / d c_w
        J.p[0] = jcv; J.p[1] = gk; J.p[2] = jcw; J.p[3] = -gk;
        J.c[0] = gD + tF * jcv; J.c[1] = tF * gk; J.c[2] = -gD + tF * jcw; J.c[3] = -tF * gk;
        return true;
    }
    if (lv == lw && (lv == PG || lv == PK)) {
        T gD = T(P.gD[lv]), gs = T(P.gsig[lv][lw]);
        J.c[0] = gD; J.c[2] = -gD;
        J.p[1] = gs; J.p[3] = -gs;
        return true;
    }
    if (is_conductor(lv) && is_conductor(lw)) {
        T gs = T(P.gsig[lv][lw]);
        J.p[1] = gs; J.p[3] = -gs;
        return true;
    }
    return !((lw == PE && (lv == PG || lv == PK || lv == PL)) || (lv == PE && (lw == PG || lw == PK || lw == PL)));
}

// J of one face with the interface partials of face i taken from the stored
// linearisation icoef[6][NI] (i_eta, ip_eta, i_cs, i_ce, ip_ce, ip_n)
template <class T>
__device__ inline void face_jacobian_lin(const ParT<T>& P, int lv, int lw, T cv, T cw, const float* __restrict__ icoef,
                                         int64_t NI, int64_t i, FaceJac<T>& J) {
#pragma unroll
    for (int k = 0; k < 5; ++k) { J.c[k] = T(0); J.p[k] = T(0); J.n[k] = T(0); }
    if (face_jacobian_bulk<T>(P, lv, lw, cv, cw, J)) return;
    const T i_eta = T(icoef[i]), ip_eta = T(icoef[NI + i]), i_cs = T(icoef[2 * NI + i]);
    const T i_ce = T(icoef[3 * NI + i]), ip_ce = T(icoef[4 * NI + i]), ip_n = T(icoef[5 * NI + i]);
    const bool solid_side = lw == PE;
    face_jacobian_iface<T>(P, solid_side, (solid_side ? lv : lw) != PL, i_eta, i_cs, i_ce, ip_eta, ip_ce, ip_n, J);
}

template <class T>
__device__ inline void face_jacobian(const ParT<T>& P, int lv, int lw, T cv, T pv, T cw, T pw,
                                     T nf, bool gate, T s_i0, T k_pl, FaceJac<T>& J) {
#pragma unroll
    for (int k = 0; k < 5; ++k) { J.c[k] = T(0); J.p[k] = T(0); J.n[k] = T(0); }
    if (lv == PE && lw == PE) {
        T cmin = T(P.cmin[PE]);
        T mv = cv >= cmin ? T(1) : T(0), mw = cw >= cmin ? T(1) : T(0);
        T S = tmax(cv, cmin) + tmax(cw, cmin);
        T iS = T(1) / S;
        T dc = cw - cv;
        T r = dc * iS * iS;
        T gm = T(P.E_gm), gk = T(P.E_gk), tF = T(P.E_tF), gD = T(P.E_gD);
        T jcv = gm * (iS + r * mv);       // d j / d c_v
        T jcw = -gm * (iS - r * mw);      // d j / d c_w
        J.p[0] = jcv; J.p[1] = gk; J.p[2] = jcw; J.p[3] = -gk;
        J.c[0] = gD + tF * jcv; J.c[1] = tF * gk; J.c[2] = -gD + tF * jcw; J.c[3] = -tF * gk;
    } else if (lv == lw && (lv == PG || lv == PK)) {
        T gD = T(P.gD[lv]), gs = T(P.gsig[lv][lw]);
        J.c[0] = gD; J.c[2] = -gD;
        J.p[1] = gs; J.p[3] = -gs;
    } else if (is_conductor(lv) && is_conductor(lw)) {
        T gs = T(P.gsig[lv][lw]);
        J.p[1] = gs; J.p[3] = -gs;
    } else if (lw == PE && (lv == PG || lv == PK || lv == PL)) {
        T i_eta, i_cs, i_ce, ip_eta, ip_ce, ip_n;
        interface_partials<T>(P, lv, cv, pv, cw, pw, nf, gate, s_i0, k_pl, i_eta, i_cs, i_ce,
                              ip_eta, ip_ce, ip_n);
        T A = T(P.A), AF = T(P.A) * T(P.invF);
        if (lv != PL) {
            J.c[0] = AF * i_cs; J.c[1] = AF * i_eta; J.c[2] = AF * i_ce; J.c[3] = -AF * i_eta;
        }
        J.p[0] = A * i_cs; J.p[1] = A * (i_eta + ip_eta); J.p[2] = A * (i_ce + ip_ce);
        J.p[3] = -A * (i_eta + ip_eta); J.p[4] = A * ip_n;
        T iF = T(P.invF);
        J.n[1] = iF * ip_eta; J.n[2] = iF * ip_ce; J.n[3] = -iF * ip_eta; J.n[4] = iF * ip_n;
    } else if (lv == PE && (lw == PG || lw == PK || lw == PL)) {
        T i_eta, i_cs, i_ce, ip_eta, ip_ce, ip_n;
        interface_partials<T>(P, lw, cw, pw, cv, pv, nf, gate, s_i0, k_pl, i_eta, i_cs, i_ce,
                              ip_eta, ip_ce, ip_n);
        T A = T(P.A), AF = T(P.A) * T(P.invF);
        T te = i_eta + ip_eta;
        J.c[0] = -AF * (i_ce + ip_ce); J.c[1] = AF * te; J.c[2] = -AF * i_cs; J.c[3] = -AF * te;
        J.c[4] = -AF * ip_n;
        J.p[0] = -A * (i_ce + ip_ce); J.p[1] = A * te; J.p[2] = -A * i_cs; J.p[3] = -A * te;
        J.p[4] = -A * ip_n;
        // face row i_pl/F seen from the electrolyte side: x = (c_e, phi_e, c_g, phi_g, n)
        T iF = T(P.invF);
        J.n[0] = iF * ip_ce; J.n[1] = -iF * ip_eta; J.n[3] = iF * ip_eta; J.n[4] = iF * ip_n;
    }
}

// Directional derivative of one face's contribution to v's rows, written so
// that every conduction, diffusion and overpotential coupling multiplies a
// difference of the direction's entries (g (dx_w - dx_v), i_eta (dPhi_s -
// dphi_e)).  The caller passes those differences, ddc = dc_w - dc_v (used only
// between voxels of one phase) and ddp = dphi_w - dphi_v, computed from the
// direction's full-precision storage (float-float or FP64), so that a uniform
// shift of a conductor's potential produces an exactly zero flux change and
// the weakly pinned modes (particles and electrolyte held only by
// Butler-Volmer conductances ~1e-6 of the bulk ones) survive FP32 arithmetic;
// multiplying absolute entries and subtracting would leave rounding of the
// size of those conductances.  dc_v, dc_w, dn_f enter only through terms
// without cancellation.  Also returns the diagonal entries dR_c(v)/dc_v,
// dR_phi(v)/dphi_v of this face (dgc, dgp) and, for a graphite v next to
// electrolyte w, the face row's change jn and its diagonal d(i_pl/F)/dn (jnn,
// without the 1/dt of the storage term).
// TC: precision of the state and of the nonlinear coefficients (sqrt, sinh,
// cosh, exp, OCP, divisions); TV: precision of the direction and of the
// accumulated result.
template <class TC, class TV>
__device__ inline void face_jvp(const ParT<TC>& P, int lv, int lw, TC cv, TC pv, TC cw, TC pw, TC nf, bool gate,
                                TC s_i0, TC k_pl, TV dcv, TV dcw, TV ddc, TV ddp, TV dnf, TV& jc, TV& jp, TV& jn,
                                TV& jnn, TV& dgc, TV& dgp) {
    if (lv == PE && lw == PE) {
        TC cmin = P.cmin[PE];
        TC mv = cv >= cmin ? TC(1) : TC(0), mw = cw >= cmin ? TC(1) : TC(0);
        TC S = tmax(cv, cmin) + tmax(cw, cmin);
        TC iS = TC(1) / S;
        TC dc = cw - cv;
        TC r = dc * iS * iS;
        TC gm = P.E_gm, gk = P.E_gk, tF = P.E_tF, gD = P.E_gD;
        // j = -gk dphi - gm dc/S ;  d(dc/S) = ddc/S - dc/S^2 (m_v dc_v + m_w dc_w)
        TV dj = -TV(gk) * ddp - TV(gm) * (ddc * TV(iS) - TV(r) * (TV(mv) * dcv + TV(mw) * dcw));
        jc += -TV(gD) * ddc + TV(tF) * dj;
        jp += dj;
        TC jcv = gm * (iS + r * mv);
        dgc += TV(gD + tF * jcv);
        dgp += TV(gk);
    } else if (lv == lw && (lv == PG || lv == PK)) {
        TV gD = TV(P.gD[lv]), gs = TV(P.gsig[lv][lw]);
        jc += -gD * ddc;
        jp += -gs * ddp;
        dgc += gD;
        dgp += gs;
    } else if (is_conductor(lv) && is_conductor(lw)) {
        TV gs = TV(P.gsig[lv][lw]);
        jp += -gs * ddp;
        dgp += gs;
    } else if (lw == PE && (lv == PG || lv == PK || lv == PL)) {
        TC i_eta, i_cs, i_ce, ip_eta, ip_ce, ip_n;
        interface_partials<TC>(P, lv, cv, pv, cw, pw, nf, gate, s_i0, k_pl, i_eta, i_cs, i_ce, ip_eta, ip_ce, ip_n);
        TV deta = -ddp;   // dPhi_s - dphi_e
        TV dibv = TV(i_eta) * deta + TV(i_cs) * dcv + TV(i_ce) * dcw;
        TV dipl = TV(ip_eta) * deta + TV(ip_ce) * dcw + TV(ip_n) * dnf;
        TV A = TV(P.A), AF = TV(P.A * P.invF);
        if (lv != PL) {
            jc += AF * dibv;
            dgc += AF * TV(i_cs);
        }
        jp += A * (dibv + dipl);
        dgp += A * TV(i_eta + ip_eta);
        jn = TV(P.invF) * dipl;
        jnn = TV(P.invF * ip_n);
    } else if (lv == PE && (lw == PG || lw == PK || lw == PL)) {
        TC i_eta, i_cs, i_ce, ip_eta, ip_ce, ip_n;
        interface_partials<TC>(P, lw, cw, pw, cv, pv, nf, gate, s_i0, k_pl, i_eta, i_cs, i_ce, ip_eta, ip_ce, ip_n);
        TV deta = ddp;    // dPhi_s - dphi_e with the solid at w
        TV di = TV(i_eta + ip_eta) * deta + TV(i_cs) * dcw + TV(i_ce + ip_ce) * dcv + TV(ip_n) * dnf;
        TV A = TV(P.A), AF = TV(P.A * P.invF);
        jc -= AF * di;
        jp -= A * di;
        dgc += -AF * TV(i_ce + ip_ce);
        dgp += A * TV(i_eta + ip_eta);
    }
}

}  // namespace mb
