// Continuous-batching dose server on top of the C ABI.
//
// Requests (robust scenarios of one plan over one resident 4DCT: seed,
// history count, stopping-power scale, setup shift) wait in a FIFO queue.
// Each step admits queued requests into free slots -- a slot is a view of
// the resident grid with the plan loaded once (copied from a template view
// whose delivery timeline ran at server creation), created while the memory
// budget allows and reused afterwards -- then gives every active request a
// share of the step's history budget over its phases and runs all those
// slices in ONE persistent launch (dose_run_batch).  A request whose last
// slice ran is finished (normalised, accumulated onto the reference phase)
// and reported.  Requests that arrive while others are running join at the
// next step, so short requests are not stuck behind long ones, and their
// work shares launches with everything else in flight.  Because histories
// are keyed by (seed, history, phase), a request's result does not depend
// on the mix it was served in.
#include <cuda_runtime.h>
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "dose.h"
#include "kernels.h"

static_assert(sizeof(dose_server_config) == 64, "ABI layout");

struct dose_server {
    struct Queued {
        int64_t id;
        dose_request req;
        bool own_delivery;             // req.delivery was given (copied into dlv)
        dose_delivery dlv;
    };
    struct Slot {
        dose_ctx *view = nullptr;
        int64_t request = -1;          // -1: free
        bool loaded_own = false;       // the plan is loaded with loaded_dlv, not the server's
        dose_delivery loaded_dlv{};
    };
    struct Active {
        int64_t id;
        dose_request req;
        int slot;
        std::vector<int> phases;       // phases the request's delivery reaches
        uint64_t per_phase;            // histories per phase with protons
        uint64_t next;                 // next history index (same for every phase)
        uint32_t waited = 0;           // steps in a row without a slice
    };
    dose_ctx *base = nullptr;
    dose_ctx *tmpl = nullptr;          // a view with the plan and the server's delivery loaded
    dose_server_config cfg{};
    std::vector<dose_spot> spots;
    dose_delivery delivery{};
    bool has_delivery = false;
    std::vector<int> phases;           // phases whose subplan has protons
    size_t slot_bytes = 0;
    std::vector<Slot> slots;
    std::deque<Queued> queue;
    std::vector<Active> active;
    std::vector<int64_t> done;         // finished, result not yet released
    std::vector<std::pair<int64_t, int>> finished_slot;  // id -> slot
    int64_t next_id = 0;
    uint64_t histories_done = 0, completed = 0, steps = 0;
    // timing of the steps (seconds): batch and accumulation on the device,
    // the step on the host; events reused by every step
    double t_batch = 0.0, t_accum = 0.0, t_wall = 0.0;
    uint64_t timed_steps = 0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    std::string err;
};

namespace {

int sfail(dose_server *s, int code, const char *msg)
{
    if (s) s->err = msg;
    dose::set_thread_error(msg);
    return code;
}

// Device bytes one slot holds: tallies, doses and ledgers of every phase,
// the EMTM E/M arrays and interleaved-field scratch, the accumulated dose,
// the per-phase allocation arrays and the plan (an upper bound, rounded up).
size_t slot_footprint(int nx, int ny, int nz, int n_phases, int64_t n_spots, bool accumulate)
{
    const size_t nvox = (size_t)nx * ny * nz, P = (size_t)n_phases;
    size_t b = P * nvox * (8 + 4) + P * 64;
    if (accumulate) b += 2 * P * nvox * 8 + nvox * 4 + P * 4 + 64 + nvox * 4 + nvox * 16 + P * 48;
    b += P * (size_t)(n_spots + 1) * (8 + 4 + 8) + (size_t)n_spots * (16 + 8 + 4 + 4 + 8 * P) + (1 << 20);
    return b;
}

}  // namespace

extern "C" {

int dose_server_create(dose_ctx *base, const dose_server_config *cfg, const dose_spot *spots, int64_t n_spots,
                       const dose_delivery *delivery, dose_server **out)
{
    if (!out) return sfail(nullptr, DOSE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!base || !cfg || !spots || n_spots <= 0) return sfail(nullptr, DOSE_EINVAL, "base, cfg and spots are required");
    if (cfg->step_histories == 0) return sfail(nullptr, DOSE_EINVAL, "step_histories must be positive");
    if (cfg->accumulate && (cfg->nsub[0] < 1 || cfg->nsub[1] < 1 || cfg->nsub[2] < 1))
        return sfail(nullptr, DOSE_EINVAL, "nsub must be positive");
    if (cfg->policy != DOSE_SERVE_FAIR && cfg->policy != DOSE_SERVE_SHORTEST_FIRST)
        return sfail(nullptr, DOSE_EINVAL, "policy must be DOSE_SERVE_FAIR or DOSE_SERVE_SHORTEST_FIRST");
    if (cfg->max_wait_steps < 0) return sfail(nullptr, DOSE_EINVAL, "max_wait_steps must be 0 or positive");
    dose_server *s = new dose_server;
    s->base = base;
    s->cfg = *cfg;
    s->spots.assign(spots, spots + n_spots);
    if (delivery) { s->delivery = *delivery; s->has_delivery = true; }
    // the base carries the grid; a template view holds the plan with the
    // server's delivery (the timeline runs once: slots copy its result) and
    // gives the phases the plan reaches
    int rc = dose_create_view(base, &s->tmpl);
    if (rc) { delete s; return rc; }
    rc = dose_add_spots(s->tmpl, spots, n_spots, delivery, nullptr);
    int dims[4] = {0, 0, 0, 0};
    if (!rc) dose::grid_info(s->tmpl, dims);
    std::vector<uint64_t> pp;
    if (!rc) {
        pp.resize((size_t)dims[3] * n_spots);
        rc = dose_read(s->tmpl, DOSE_SUBPLAN, 0, pp.data(), pp.size() * 8, 0, nullptr);
    }
    if (rc) { dose_destroy(s->tmpl); delete s; return rc; }
    for (int p = 0; p < dims[3]; ++p) {
        uint64_t w = 0;
        for (int64_t k = 0; k < n_spots; ++k) w += pp[(size_t)p * n_spots + k];
        if (w) s->phases.push_back(p);
    }
    if (s->phases.empty()) {
        dose_destroy(s->tmpl);
        delete s;
        return sfail(nullptr, DOSE_EINVAL, "the plan delivers no protons");
    }
    s->slot_bytes = slot_footprint(dims[0], dims[1], dims[2], dims[3], n_spots, cfg->accumulate != 0);
    if (cfg->memory_budget_bytes < s->slot_bytes) {
        dose_destroy(s->tmpl);
        delete s;
        return sfail(nullptr, DOSE_EINVAL, "memory budget is smaller than one request slot");
    }
    *out = s;
    return DOSE_OK;
}

int dose_server_submit(dose_server *s, const dose_request *req, int64_t *id)
{
    if (!s || !req) return sfail(s, DOSE_EINVAL, "server and request are required");
    if (req->n_histories == 0) return sfail(s, DOSE_EINVAL, "request has no histories");
    const int64_t rid = s->next_id++;
    dose_server::Queued q;
    q.id = rid;
    q.req = *req;
    q.own_delivery = req->delivery != nullptr;
    if (q.own_delivery) q.dlv = *req->delivery;
    q.req.delivery = nullptr;                      // the copy in q.dlv is used
    s->queue.push_back(q);
    if (id) *id = rid;
    return DOSE_OK;
}

int dose_server_step(dose_server *s, void *stream, int64_t *completed, int max_completed, int *n_completed)
{
    if (!s) return sfail(s, DOSE_EINVAL, "server is NULL");
    if (n_completed) *n_completed = 0;
    const size_t max_slots = std::max<size_t>(1, s->cfg.memory_budget_bytes / s->slot_bytes);
    const size_t cap = s->cfg.max_active > 0 ? std::min<size_t>(max_slots, (size_t)s->cfg.max_active) : max_slots;
    // admit: free slots first, then new slots while the budget allows
    while (!s->queue.empty()) {
        int slot = -1;
        for (size_t k = 0; k < s->slots.size(); ++k)
            if (s->slots[k].request < 0) { slot = (int)k; break; }
        const dose_server::Queued &q = s->queue.front();
        if (slot < 0 && s->slots.size() < cap) {
            dose_server::Slot sl;
            int rc = dose_create_view(s->base, &sl.view);
            if (!rc) rc = dose::copy_plan(sl.view, s->tmpl, stream);
            if (rc) {
                if (sl.view) dose_destroy(sl.view);
                if (rc == DOSE_ENOMEM) break;            // no room now; retry next step
                return rc;
            }
            s->slots.push_back(sl);
            slot = (int)s->slots.size() - 1;
        }
        if (slot < 0) break;
        dose_server::Slot &sl = s->slots[slot];
        dose_server::Active a;
        a.id = q.id;
        a.req = q.req;
        a.slot = slot;
        a.phases = s->phases;
        // a request with its own delivery reloads the slot's plan with it
        // (the slot keeps it for the next request with the same delivery)
        const bool want_own = q.own_delivery;
        const bool same = want_own ? (sl.loaded_own && std::memcmp(&sl.loaded_dlv, &q.dlv, sizeof q.dlv) == 0)
                                   : !sl.loaded_own;
        if (!same) {
            int rc = want_own ? dose_add_spots(sl.view, s->spots.data(), (int64_t)s->spots.size(), &q.dlv, stream)
                              : dose::copy_plan(sl.view, s->tmpl, stream);
            if (rc) return rc;
            sl.loaded_own = want_own;
            if (want_own) sl.loaded_dlv = q.dlv;
        }
        if (want_own) {
            int dims[4] = {0, 0, 0, 0};
            dose::grid_info(sl.view, dims);
            const int64_t S = (int64_t)s->spots.size();
            std::vector<uint64_t> pp((size_t)dims[3] * S);
            int rc = dose_read(sl.view, DOSE_SUBPLAN, 0, pp.data(), pp.size() * 8, 0, stream);
            if (rc) return rc;
            a.phases.clear();
            for (int p = 0; p < dims[3]; ++p) {
                uint64_t w = 0;
                for (int64_t k = 0; k < S; ++k) w += pp[(size_t)p * S + k];
                if (w) a.phases.push_back(p);
            }
        }
        a.per_phase = a.phases.empty() ? 0 : std::max<uint64_t>(1, a.req.n_histories / a.phases.size());
        a.next = 0;
        sl.request = a.id;
        s->queue.pop_front();
        s->active.push_back(a);
    }
    if (s->active.empty()) return DOSE_OK;
    const auto wall0 = std::chrono::steady_clock::now();
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    if (!s->ev[0])
        for (auto &e : s->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return sfail(s, DOSE_ECUDA, "cudaEventCreate failed");
    // the step's histories: an equal share for every active request, or
    // (DOSE_SERVE_SHORTEST_FIRST) the budget handed out in order of the
    // histories each request has left, fewest first, after the requests
    // that have waited max_wait_steps; a request left without a slice
    // waits for the next step.  A slice has at least min_slice histories
    // per phase, so every slice makes progress.
    size_t phase_jobs = 0;
    for (const auto &a : s->active) phase_jobs += a.phases.size();
    const uint64_t min_slice = s->cfg.min_slice ? s->cfg.min_slice : 1;
    std::vector<uint64_t> take(s->active.size(), 0);           // histories per phase this step
    if (s->cfg.policy == DOSE_SERVE_SHORTEST_FIRST) {
        std::vector<size_t> order(s->active.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        auto left = [&](size_t i) {
            const auto &a = s->active[i];
            return (a.per_phase - a.next) * (uint64_t)a.phases.size();
        };
        // a request that has waited max_wait_steps steps goes first and
        // gets at least min_slice even when the budget is spent
        const uint32_t bound = (uint32_t)s->cfg.max_wait_steps;
        auto overdue = [&](size_t i) { return bound > 0 && s->active[i].waited >= bound; };
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
            const bool ox = overdue(x), oy = overdue(y);
            return ox != oy ? ox : left(x) < left(y);
        });
        uint64_t budget = s->cfg.step_histories;
        for (size_t i : order) {
            const auto &a = s->active[i];
            if (a.phases.empty() || (budget == 0 && !overdue(i))) continue;
            const uint64_t nph = a.phases.size();
            const uint64_t t = std::min(a.per_phase - a.next, std::max(min_slice, budget / nph));
            take[i] = t;
            budget = budget > t * nph ? budget - t * nph : 0;
        }
    } else {
        const uint64_t share = std::max<uint64_t>(min_slice, s->cfg.step_histories / std::max<size_t>(1, phase_jobs));
        for (size_t i = 0; i < s->active.size(); ++i)
            take[i] = std::min(s->active[i].per_phase - s->active[i].next, share);
    }
    std::vector<dose_job> jobs;
    std::vector<int> finishing;
    for (size_t i = 0; i < s->active.size(); ++i) {
        auto &a = s->active[i];
        if (a.phases.empty()) {                      // nothing delivered: a zero dose
            finishing.push_back((int)i);
            continue;
        }
        if (take[i] == 0) {                          // waits for a later step
            ++a.waited;
            continue;
        }
        a.waited = 0;
        const uint64_t end = a.next + take[i];
        for (int p : a.phases) {
            dose_job j;
            j.ctx = s->slots[a.slot].view;
            j.phase = p;
            j.flags = (a.next == 0 ? DOSE_JOB_CLEAR : 0u) | (end == a.per_phase ? DOSE_JOB_FINISH : 0u);
            j.n_histories = a.per_phase;
            j.hist_begin = a.next;
            j.hist_end = end;
            j.seed = a.req.seed;
            j.spr_scale = a.req.spr_scale;
            for (int k = 0; k < 3; ++k) j.shift_mm[k] = a.req.shift_mm[k];
            jobs.push_back(j);
        }
        s->histories_done += (end - a.next) * a.phases.size();
        a.next = end;
        if (end == a.per_phase) finishing.push_back((int)i);
    }
    cudaEventRecord(s->ev[0], cs);
    int rc = jobs.empty() ? DOSE_OK : dose_run_batch(jobs.data(), (int)jobs.size(), stream);
    if (rc) return rc;
    cudaEventRecord(s->ev[1], cs);
    for (int i : finishing) {
        auto &a = s->active[i];
        dose_ctx *v = s->slots[a.slot].view;
        int dims[4];
        dose::grid_info(v, dims);
        // phases the request's delivery does not reach carry zero dose
        for (int p = 0; p < dims[3]; ++p)
            if (std::find(a.phases.begin(), a.phases.end(), p) == a.phases.end())
                if ((rc = dose::set_phase_zero(v, p, stream))) return rc;
        if (s->cfg.accumulate &&
            (rc = dose_accumulate_subvoxel(v, s->cfg.ref_phase, s->cfg.nsub, s->cfg.dvf, 1, nullptr, 0, 0, stream)))
            return rc;
    }
    cudaEventRecord(s->ev[2], cs);
    cudaError_t e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return sfail(s, DOSE_ECUDA, cudaGetErrorString(e));
    float ms_batch = 0.0f, ms_accum = 0.0f;
    if (cudaEventElapsedTime(&ms_batch, s->ev[0], s->ev[1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms_accum, s->ev[1], s->ev[2]) == cudaSuccess) {
        s->t_batch += 1e-3 * ms_batch;
        s->t_accum += 1e-3 * ms_accum;
        ++s->timed_steps;
    }
    cudaGetLastError();
    s->t_wall += std::chrono::duration<double>(std::chrono::steady_clock::now() - wall0).count();
    ++s->steps;
    std::vector<dose_server::Active> keep;
    int nc = 0;
    for (size_t i = 0; i < s->active.size(); ++i) {
        const bool fin = std::find(finishing.begin(), finishing.end(), (int)i) != finishing.end();
        if (!fin) { keep.push_back(s->active[i]); continue; }
        s->done.push_back(s->active[i].id);
        s->finished_slot.emplace_back(s->active[i].id, s->active[i].slot);
        ++s->completed;
        if (completed && nc < max_completed) completed[nc] = s->active[i].id;
        ++nc;
    }
    s->active.swap(keep);
    if (n_completed) *n_completed = std::min(nc, max_completed);
    return DOSE_OK;
}

int dose_server_result(dose_server *s, int64_t id, int what, int phase, void *dst, size_t bytes, int dst_on_device,
                       void *stream)
{
    if (!s) return sfail(s, DOSE_EINVAL, "server is NULL");
    for (auto &f : s->finished_slot)
        if (f.first == id)
            return dose_read(s->slots[f.second].view, what, phase, dst, bytes, dst_on_device, stream);
    return sfail(s, DOSE_ESTATE, "request is not finished or was released");
}

int dose_server_release(dose_server *s, int64_t id)
{
    if (!s) return sfail(s, DOSE_EINVAL, "server is NULL");
    for (size_t k = 0; k < s->finished_slot.size(); ++k) {
        if (s->finished_slot[k].first != id) continue;
        s->slots[s->finished_slot[k].second].request = -1;
        s->finished_slot.erase(s->finished_slot.begin() + k);
        s->done.erase(std::remove(s->done.begin(), s->done.end(), id), s->done.end());
        return DOSE_OK;
    }
    return sfail(s, DOSE_ESTATE, "request is not finished or was released");
}

int dose_server_stats(const dose_server *s, uint64_t out[8])
{
    if (!s || !out) return sfail(nullptr, DOSE_EINVAL, "server and out are required");
    out[0] = s->queue.size();
    out[1] = s->active.size();
    out[2] = s->slots.size();
    out[3] = s->completed;
    out[4] = s->histories_done;
    out[5] = s->steps;
    out[6] = s->slot_bytes;
    out[7] = s->done.size();
    return DOSE_OK;
}

int dose_server_timing(const dose_server *s, double out[4])
{
    if (!s || !out) return sfail(nullptr, DOSE_EINVAL, "server and out are required");
    out[0] = s->t_batch;
    out[1] = s->t_accum;
    out[2] = s->t_wall;
    out[3] = (double)s->timed_steps;
    return DOSE_OK;
}

void dose_server_destroy(dose_server *s)
{
    if (!s) return;
    for (auto &e : s->ev)
        if (e) cudaEventDestroy(e);
    for (auto &sl : s->slots) dose_destroy(sl.view);
    dose_destroy(s->tmpl);
    delete s;
}

}  // extern "C"
