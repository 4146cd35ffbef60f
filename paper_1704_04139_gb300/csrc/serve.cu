// serve.cu -- serving loop for parameter-study queries: continuous batching
// of reduced-model requests in a resident slot batch (one step per launch
// round, admission and retirement at step boundaries) and full-order
// validation solves on worker threads with their own cells and streams,
// admitted by device memory.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mb_internal.h"

namespace {

struct Req {
    uint64_t ticket = 0;
    mb_request r{};
    double t_submit = 0, t_start = 0, t_done = 0;
    int status = MB_EPENDING;
    bool done = false;
    std::vector<double> V, S;
};

}  // namespace

struct mb_server {
    mb_serve_opts o{};
    std::vector<uint8_t> labels;
    mb_params prm{};
    mb_solver_opts fopts{};
    bool has_fom = false;
    int device = 0;
    std::mutex m;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Req>> rom_q, fom_q;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> reqs;
    uint64_t next = 1;
    bool stop = false;
    int64_t fom_bytes = 0;         // device memory of running full-order cells
    int64_t fom_cell_bytes = 0;    // per cell (measured on the first one)
    bool measuring = false;        // a worker is creating the first cell (its size is not known yet)
    int fom_cells = 0, fom_cells_peak = 0;   // full-order cells alive now / at most
    std::thread rom_thread;
    std::vector<std::thread> fom_threads;
    std::chrono::steady_clock::time_point t0;
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void finish(mb_server* S, const std::shared_ptr<Req>& q, int status) {
    q->status = status;
    q->t_done = S->now();
    q->done = true;
}

void rom_loop(mb_server* S) {
    cudaSetDevice(S->device);
    mb_rom* R = S->o.rom;
    const int B = S->o.rom_slots;
    if (mb::rom_batch_alloc(R, B)) {
        std::lock_guard<std::mutex> lk(S->m);
        for (auto& q : S->rom_q) finish(S, q, MB_ENOMEM);
        S->rom_q.clear();
        return;
    }
    std::vector<std::shared_ptr<Req>> slot(B);
    std::vector<double> hV(B), hS(B);
    std::vector<int> hf(B);
    for (;;) {
        std::vector<int> started;
        {
            std::unique_lock<std::mutex> lk(S->m);
            auto busy = [&]() {
                for (auto& q : slot)
                    if (q) return true;
                return false;
            };
            S->cv.wait(lk, [&]() { return S->stop || !S->rom_q.empty() || busy(); });
            if (S->stop) break;
            for (int b = 0; b < B && !S->rom_q.empty(); ++b) {
                if (slot[b]) continue;
                slot[b] = S->rom_q.front();
                S->rom_q.pop_front();
                slot[b]->t_start = S->now();
                started.push_back(b);
            }
        }
        int rc = MB_OK;
        for (int b : started)
            if (!rc) rc = mb::rom_slot_start(R, b, slot[b]->r.prm, slot[b]->r.dt);
        if (!rc && !started.empty()) rc = mb::rom_batch_outputs(R, hV.data(), hS.data(), hf.data());
        if (!rc) {
            std::lock_guard<std::mutex> lk(S->m);
            for (int b : started) {
                slot[b]->V.push_back(hV[b]);
                slot[b]->S.push_back(hS[b]);
                if (slot[b]->r.n_steps == 0) {
                    finish(S, slot[b], MB_OK);
                    mb::rom_slot_clear(R, b);
                    slot[b].reset();
                }
            }
        }
        bool any = false;
        for (auto& q : slot) any |= (bool)q;
        if (!rc && any) rc = mb::rom_batch_step(R);
        if (!rc && any) rc = mb::rom_batch_outputs(R, hV.data(), hS.data(), hf.data());
        std::lock_guard<std::mutex> lk(S->m);
        for (int b = 0; b < B; ++b) {
            if (!slot[b]) continue;
            auto& q = slot[b];
            if (rc) {
                finish(S, q, rc);
            } else if (hf[b]) {
                finish(S, q, MB_ENOCONV);
            } else {
                q->V.push_back(hV[b]);
                q->S.push_back(hS[b]);
                if ((int)q->V.size() == q->r.n_steps + 1) finish(S, q, MB_OK);
                else if (q->r.v_cutoff > 0.0 && hV[b] >= q->r.v_cutoff) finish(S, q, MB_ECUTOFF);
            }
            if (q->done) {
                mb::rom_slot_clear(R, b);
                slot[b].reset();
            }
        }
    }
}

double cell_potential(mb_cell* c) {
    std::vector<double> u(c->n);
    if (mb_state_get(c, u.data())) return NAN;
    const int64_t N = c->D.N, last0 = (int64_t)(c->D.nt - 1) * c->D.syz;
    double s = 0.0;
    for (int64_t v = last0; v < N; ++v) s += u[N + v];
    return s / (double)(N - last0);
}

// A worker keeps the cell it created for its first request and resets its
// state for the next ones (no device allocation or release, which would
// synchronise the device, in steady state).  A worker without a cell is
// admitted while the cells' device memory stays within the budget; until the
// first cell has been created and measured, only one worker at a time may
// create one (its size is charged once known), and one cell is always allowed.
bool fom_admit(const mb_server* S, bool has_cell) {
    if (has_cell) return true;
    if (S->measuring) return false;
    if (S->fom_cells == 0) return true;
    if (S->fom_cell_bytes == 0) return false;
    return S->fom_bytes + S->fom_cell_bytes <= S->o.fom_budget_bytes;
}

void fom_loop(mb_server* S) {
    cudaSetDevice(S->device);
    mb_cell* c = nullptr;
    int64_t charged = 0;   // this worker's share of fom_bytes
    for (;;) {
        std::shared_ptr<Req> q;
        bool measure = false;
        {
            std::unique_lock<std::mutex> lk(S->m);
            S->cv.wait(lk, [&]() { return S->stop || (!S->fom_q.empty() && fom_admit(S, c != nullptr)); });
            if (S->stop) break;
            q = S->fom_q.front();
            S->fom_q.pop_front();
            if (!c) {
                measure = S->fom_cell_bytes == 0;
                if (measure) S->measuring = true;
                charged = S->fom_cell_bytes;
                S->fom_bytes += charged;
                S->fom_cells += 1;
                if (S->fom_cells > S->fom_cells_peak) S->fom_cells_peak = S->fom_cells;
            }
            q->t_start = S->now();
        }
        int rc = MB_OK;
        if (!c) {
            rc = mb_cell_create(S->labels.data(), S->o.nt, S->o.ny, S->o.nz, S->o.h, &S->prm, &S->fopts, &c);
            {
                std::lock_guard<std::mutex> lk(S->m);
                if (!rc) {
                    mb_cell_info info;
                    mb_cell_info_get(c, &info);
                    if (!S->fom_cell_bytes) S->fom_cell_bytes = info.device_bytes;
                    S->fom_bytes += info.device_bytes - charged;
                    charged = info.device_bytes;
                } else {
                    c = nullptr;
                    S->fom_bytes -= charged;
                    S->fom_cells -= 1;
                    charged = 0;
                }
                if (measure) S->measuring = false;
            }
            S->cv.notify_all();
        } else {
            rc = mb::launch_init_state(c, c->u);
            if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess)
                rc = mb::cuda_fail(cudaGetLastError(), "fom reset");
        }
        if (!rc) rc = mb_cell_set_scales(c, q->r.prm.s_i0, q->r.prm.k_pl);
        if (!rc) {
            q->V.push_back(cell_potential(c));
            q->S.push_back(NAN);
        }
        for (int k = 0; !rc && k < q->r.n_steps; ++k) {
            mb_step_info info;
            rc = mb_step(c, q->r.dt, q->r.prm.I_app, &info);
            if (!rc) {
                q->V.push_back(info.V_cell);
                q->S.push_back(info.mean_c_solid);
                if (q->r.v_cutoff > 0.0 && info.V_cell >= q->r.v_cutoff && k + 1 < q->r.n_steps) {
                    rc = MB_ECUTOFF;
                    break;
                }
            }
        }
        {
            std::lock_guard<std::mutex> lk(S->m);
            finish(S, q, rc);
        }
        S->cv.notify_all();
    }
    if (c) {
        mb_cell_destroy(c);
        std::lock_guard<std::mutex> lk(S->m);
        S->fom_bytes -= charged;
        S->fom_cells -= 1;
    }
}

}  // namespace

using namespace mb;

extern "C" int mb_serve_create(const mb_serve_opts* o, mb_server** out) {
    if (!o || !out || o->rom_slots < 1 || o->fom_workers < 1 || (!o->rom && !o->fom_labels) ||
        (o->fom_labels && (!o->params || o->nt < 1 || o->ny < 1 || o->nz < 1 || !(o->h > 0)))) {
        set_error("mb_serve_create: invalid argument");
        return MB_EINVAL;
    }
    mb_server* S = new mb_server();
    S->o = *o;
    S->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&S->device);
    if (o->fom_labels) {
        S->has_fom = true;
        S->labels.assign(o->fom_labels, o->fom_labels + (size_t)o->nt * o->ny * o->nz);
        S->prm = *o->params;
        if (o->fom_opts) S->fopts = *o->fom_opts;
        else mb_opts_default(&S->fopts);
    }
    if (o->rom) S->rom_thread = std::thread(rom_loop, S);
    if (S->has_fom)
        for (int i = 0; i < o->fom_workers; ++i) S->fom_threads.emplace_back(fom_loop, S);
    *out = S;
    return MB_OK;
}

extern "C" int mb_serve_submit(mb_server* S, const mb_request* r, uint64_t* ticket) {
    if (!S || !r || !ticket || r->n_steps < 0 || !(r->dt > 0) || (r->kind != MB_REQ_ROM && r->kind != MB_REQ_FOM) ||
        (r->kind == MB_REQ_ROM && !S->o.rom) || (r->kind == MB_REQ_FOM && !S->has_fom)) {
        set_error("mb_serve_submit: invalid request");
        return MB_EINVAL;
    }
    auto q = std::make_shared<Req>();
    q->r = *r;
    {
        std::lock_guard<std::mutex> lk(S->m);
        q->ticket = S->next++;
        q->t_submit = S->now();
        S->reqs[q->ticket] = q;
        (r->kind == MB_REQ_ROM ? S->rom_q : S->fom_q).push_back(q);
        *ticket = q->ticket;
    }
    S->cv.notify_all();
    return MB_OK;
}

extern "C" int mb_serve_poll(mb_server* S, uint64_t ticket, mb_result* out) {
    if (!S || !out) { set_error("mb_serve_poll: invalid argument"); return MB_EINVAL; }
    std::shared_ptr<Req> q;
    {
        std::lock_guard<std::mutex> lk(S->m);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) { set_error("mb_serve_poll: unknown ticket"); return MB_EINVAL; }
        q = it->second;
        if (!q->done) return MB_EPENDING;
        S->reqs.erase(it);
    }
    out->status = q->status;
    out->n_steps = (int)q->V.size() - 1;
    out->t_submit = q->t_submit;
    out->t_start = q->t_start;
    out->t_done = q->t_done;
    for (size_t k = 0; k < q->V.size(); ++k) {
        if (out->V) out->V[k] = q->V[k];
        if (out->s_ac) out->s_ac[k] = q->S[k];
    }
    return MB_OK;
}

extern "C" int mb_serve_destroy(mb_server* S) {
    if (!S) { set_error("mb_serve_destroy: invalid argument"); return MB_EINVAL; }
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->rom_thread.joinable()) S->rom_thread.join();
    for (auto& t : S->fom_threads)
        if (t.joinable()) t.join();
    delete S;
    return MB_OK;
}

// ------------------------------------------------------------ test hooks
extern "C" int mb_debug_serve_cells(mb_server* S, int* alive, int* peak, int64_t* cell_bytes) {
    if (!S || !alive || !peak || !cell_bytes) { set_error("mb_debug_serve_cells: invalid argument"); return MB_EINVAL; }
    std::lock_guard<std::mutex> lk(S->m);
    *alive = S->fom_cells;
    *peak = S->fom_cells_peak;
    *cell_bytes = S->fom_cell_bytes;
    return MB_OK;
}
