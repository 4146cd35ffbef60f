// mb_internal.h -- host-side structures shared by the libmb translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/mb.h"
#include "mb_df.cuh"
#include "mb_model.cuh"

namespace mb {

void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define MB_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::mb::cuda_fail(e_, #call);       \
    } while (0)

#define MB_CUDA_LAUNCH(what)                                            \
    do {                                                                \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return ::mb::cuda_fail(e_, what);        \
    } while (0)

// Device buffer owned by a cell.
struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct Precond;   // multigrid preconditioner (precond.cu)
struct Krylov;    // FGMRES workspace (solver.cu)

// Kernel timing and launch counting (mb_prof_* in the C-ABI).  When enabled,
// launches of the timed kernel classes are bracketed by CUDA events recorded
// on the launching stream; every kernel launch of the library increments the
// cell's launch counter whether or not timing is enabled.
enum ProfKernel { PROF_JVP = 0, PROF_RESIDUAL = 1, PROF_PRECOND = 2, PROF_SMOOTH = 3, PROF_LSMOOTH = 4,
                  PROF_NKERNELS = 5 };
struct ProfPair {
    cudaEvent_t e0, e1;
    int kind;
};
struct Prof {
    bool enabled = false;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> rec[PROF_NKERNELS];
    size_t used = 0;
    // While a CUDA graph is captured, timed launches record dedicated events
    // (graph nodes) into *capture; their times are harvested into acc_* after
    // each execution of the graph.
    std::vector<ProfPair>* capture = nullptr;
    double acc_ms[PROF_NKERNELS] = {};
    int64_t acc_n[PROF_NKERNELS] = {};
    cudaEvent_t get();
};

// Interface partial derivatives stored per interface face (structure of
// arrays, entry k of face i at [k * NI + i]): d i_bv/d eta, d i_pl/d eta,
// d i_bv/d c_s, d i_bv/d c_e, d i_pl/d c_e, d i_pl/d n (A/m^2 per unit).
constexpr int NCOEF = 6;

// plated-Li inventory (relative to the critical layer n_c) below which the
// plating gate treats a face as bare
constexpr double GATE_N_REL = 1e-9;

// Reduction scratch (deterministic two-pass reductions).
constexpr int RED_BLOCKS = 1216;      // 8 x 152 SMs
constexpr int RED_THREADS = 256;

}  // namespace mb

struct mb_cell {
    int device = 0;
    cudaStream_t stream = nullptr;
    mb::Dims D{};
    mb::DevParams P{};
    mb::DevParamsF Pf{};           // FP32 copy of P for the FP32 kernels
    mb_params prm{};
    mb_solver_opts opt{};
    double s_i0 = 1.0, k_pl = 1.0;
    double i_1c = 0.0;
    int64_t count[6] = {0, 0, 0, 0, 0, 0};
    int64_t n = 0;                 // unknowns 2N + F
    int64_t device_bytes = 0;
    std::vector<mb::DBuf> owned;

    // geometry
    uint32_t* vcode = nullptr;     // N
    uint16_t* zperm = nullptr;     // N: per z-line, the z of its voxels grouped by phase and interface
                                   //   contact (the thread order of the divergent stencil kernels)
    int32_t* if_s = nullptr;       // NI: solid voxel of each interface face
    int32_t* if_e = nullptr;       // NI: electrolyte voxel of each interface face
    int32_t* pf_g = nullptr;       // F (= if_s: plating faces come first)
    int32_t* pf_e = nullptr;       // F (= if_e)
    int8_t* pf_dir = nullptr;      // F

    // state and Newton work (FP64)
    double* u = nullptr;           // n
    double* u_old = nullptr;       // n
    double* u_pass = nullptr;      // n (start of the step, kept across halvings)
    double* r = nullptr;           // n
    double* du = nullptr;          // n
    uint8_t* gate = nullptr;       // F
    uint8_t* gate2 = nullptr;      // F
    double* red = nullptr;         // RED_BLOCKS * 64 partials
    double* red_out = nullptr;     // 64 results
    double* h_red = nullptr;       // pinned host copy of results (64)

    // mixed precision copies
    float* u32 = nullptr;          // n (linearisation point)
    float* icoef = nullptr;        // NCOEF x NI interface partials at the linearisation point
    double* icur = nullptr;        // 2 x NI interface currents (Butler-Volmer, plating) of the residual
    float* d_dtinv = nullptr;      // per-solve scalars of the stencil JVP (1/dt and row scales)
    float* rowdiag = nullptr;      // n: |diagonal| of the scaled Jacobian rows (Krylov equilibration)
    float* rowinv = nullptr;       // n: 1 / rowdiag

    mb::Precond* pc = nullptr;
    mb::Krylov* kd = nullptr;

    // adaptive time stepping (mb_step_adaptive): the state before the last
    // accepted adaptive step and that step's size; allocated at the first call
    double* u_hist = nullptr;      // n
    double* u_save = nullptr;      // n (start of the step being tried)
    bool has_hist = false;
    double dt_hist = 0.0;

    mb::Prof prof;
    int64_t launches = 0;          // kernel launches issued by the library for this cell

    // snapshot recording for the reduced-model build: when set, every Newton
    // iterate and its plating gates are appended (host copies)
    std::vector<std::vector<double>>* snap_u = nullptr;
    std::vector<std::vector<uint8_t>>* snap_g = nullptr;
};

namespace mb {
// parameter table in the arithmetic type of a kernel
template <class T> inline const ParT<T>& cell_par(const mb_cell* c);
template <> inline const ParT<double>& cell_par<double>(const mb_cell* c) { return c->P; }
template <> inline const ParT<float>& cell_par<float>(const mb_cell* c) { return c->Pf; }

// count n launches; bracket timed launches with events when profiling is on
inline void count_launch(mb_cell* c, int n = 1) { c->launches += n; }
// While a graph is captured the events are always recorded (as graph nodes),
// so that one graph serves with profiling on and off.
inline void prof_begin(mb_cell* c, cudaStream_t s, cudaEvent_t* ev) {
    *ev = nullptr;
    if (c->prof.capture) {
        // an external record node: the event is recorded each time the graph runs
        cudaEventCreate(ev);
        cudaEventRecordWithFlags(*ev, s, cudaEventRecordExternal);
    } else if (c->prof.enabled) {
        *ev = c->prof.get();
        cudaEventRecord(*ev, s);
    }
}
inline void prof_end(mb_cell* c, cudaStream_t s, int kind, cudaEvent_t ev0) {
    if ((c->prof.enabled || c->prof.capture) && ev0) {
        cudaEvent_t ev1 = nullptr;
        if (c->prof.capture) {
            cudaEventCreate(&ev1);
            cudaEventRecordWithFlags(ev1, s, cudaEventRecordExternal);
            c->prof.capture->push_back({ev0, ev1, kind});
            return;
        }
        ev1 = c->prof.get();
        cudaEventRecord(ev1, s);
        c->prof.rec[kind].push_back({ev0, ev1});
    }
}
}  // namespace mb

namespace mb {

void* cell_alloc(mb_cell* c, size_t bytes);   // cudaMalloc + bookkeeping; nullptr on failure

// ---- fom.cu launchers (all on c->stream) ----
int launch_classify(mb_cell* c, const uint8_t* d_labels);
int launch_init_state(mb_cell* c, double* u);
template <class T>
int launch_residual(mb_cell* c, const T* u, const double* u_old, const uint8_t* gate, double dt,
                    double I_app, T* r, cudaStream_t s);
// the same FP64 residual in two passes (interface currents once per face into
// c->icur, then the voxel rows): the solver's Newton residual
int launch_residual_split(mb_cell* c, const double* u, const double* u_old, const uint8_t* gate, double dt,
                          double I_app, double* r, cudaStream_t s);
// mode 0: J v;  1: S_r^-1 J S_u v (scaled units);  2: the scaled rows further divided by
// the magnitude of their diagonal entry (the row-equilibrated Krylov operator)
template <class TC, class TV>
int launch_jvp(mb_cell* c, const TC* u, const uint8_t* gate, double dt, const TV* v, TV* jv,
               cudaStream_t s, int mode = 0);
// interface partials at the linearisation point u (FP64 state in FP64, or its
// FP32 copy in FP32) into c->icoef
template <class TC>
int launch_lin_setup(mb_cell* c, const TC* u, const uint8_t* gate, cudaStream_t s);
// J v from the stored interface partials (c->icoef), the FP32 concentrations
// c->u32, the row scales c->rowdiag and 1/dt from c->d_dtinv, on a float-float
// direction v in scaled units, FP32 result; rows divided by the residual scale
// and by the row equilibration (the Krylov operator)
int launch_jvp_lin(mb_cell* c, const float2* v, float* jv, cudaStream_t s);
// c->d_dtinv = 1/dt (stream-ordered)
int set_dt(mb_cell* c, double dt, cudaStream_t s);
int launch_gate(mb_cell* c, const double* u, const double* n_old, uint8_t* gate, cudaStream_t s);
// Gates at u_old written into gate_scratch (F bytes), then the FP64 residual
// reading them, both on stream s; no profiling events, no allocation.
int launch_gate_residual_unprofiled(mb_cell* c, const double* u, const double* u_old, uint8_t* gate_scratch,
                                    double dt, double I_app, double* r, cudaStream_t s);
// inverse scales of the unknowns (which = 0: c_ref, 1, n_c) or of the
// residual rows (which = 1: V c_ref / dt or 1 for rows without c, A, n_c / dt)
struct InvScales {
    double c[6], phi, n;
};
InvScales inv_scales(const mb_cell* c, int which, double dt);
// scaled max norms: which = 0 unknown scale, 1 residual scale (needs dt)
// (out_cap, if given: the Newton step-length norm: the voxel unknowns c and phi
// in their scales and, with u_cap given, each plated inventory relative to
// max(n_c, |n_f|) of the state u_cap)
int scaled_maxnorm(mb_cell* c, const double* x, int which, double dt, double* out, double* out_cap = nullptr,
                   const double* u_cap = nullptr);
int functionals(mb_cell* c, const double* u, mb_step_info* info);
int count_diff_u8(mb_cell* c, const uint8_t* a, const uint8_t* b, int64_t n, int64_t* out);

// ---- precond.cu ----
int precond_create(mb_cell* c);
void precond_destroy(mb_cell* c);
// build at linearisation point u32 (float) for time step dt; after launch_lin_setup and set_dt of the
// same linearisation (the interface partials c->icoef carry the gates and the plated Li)
int precond_setup(mb_cell* c, const float* u32, const uint8_t* gate, double dt);
// assemble the fine smoother's stencil; after launch_lin_setup and set_dt of
// the same linearisation (it reads the interface partials and 1/dt)
int precond_setup_fine(mb_cell* c);
// z = M^{-1} r (length n, row-equilibrated Krylov units; r FP32, z float-float);
// uses the assembled fine stencil of the current linearisation.  With graph = true the
// whole application is replayed from a CUDA graph captured once per (r, z)
// buffer pair.
int precond_apply(mb_cell* c, const float* u32, const uint8_t* gate, double dt, const float* r, float2* z,
                  bool graph = true);
// add the kernel times of the last graph execution to the profile totals
void precond_harvest(mb_cell* c);
// MB_ETIMEOUT if a staged coarse sweep gave up waiting for its copies (synchronises the stream)
int precond_check(mb_cell* c);

// ---- rom.cu: slot batch of the reduced model (one step per call) ----
int rom_batch_alloc(mb_rom* R, int B);
int rom_slot_start(mb_rom* R, int b, const mb_rom_params& p, double dt);
int rom_slot_clear(mb_rom* R, int b);
int rom_batch_step(mb_rom* R);
int rom_batch_outputs(mb_rom* R, double* hV, double* hS, int* hfailed);
int rom_slot_stats(mb_rom* R, int b, long long* its, long long* flips, double* a);

// ---- solver.cu ----
int newton_step(mb_cell* c, double dt, double I_app, mb_step_info* info);
int adaptive_step(mb_cell* c, double dt_try, double I_app, const mb_adapt_opts* o, mb_adapt_info* ai,
                  mb_step_info* info);
void krylov_destroy(mb_cell* c);   // frees the host structs; buffers stay owned by the cell

}  // namespace mb
