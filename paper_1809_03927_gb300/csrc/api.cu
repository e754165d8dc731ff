// C ABI of the dose engine (include/dose.h): context management, argument
// validation and the launches of the engine's kernels.  Every step of the
// dose computation runs in the kernels; this file only checks arguments,
// owns device memory and enqueues work.
#include <cuda_runtime.h>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dose.h"
#include "engine.cuh"
#include "kernels.h"

using namespace dose;

namespace {

constexpr int kVersion = 1;
constexpr int kMaxSpots = 16384;
constexpr int kMaxFields = 64;
static_assert(sizeof(dose_delivery) == 112 && sizeof(dose_delivery_spread) == 72, "ABI layout");
constexpr int kMaxDevices = 64;

thread_local std::string g_thread_err;

struct DeviceTables {
    Tables *dev = nullptr;
    float inv_ds = 0.0f;
};
std::mutex g_tab_mutex;
DeviceTables g_tab[kMaxDevices];
Tables *g_host_tables = nullptr;
float g_host_inv_ds = 0.0f;

struct Grid {
    int n[3] = {0, 0, 0};
    float d[3] = {0, 0, 0};
    float origin[3] = {0, 0, 0};
    int n_phases = 0;
    int beam_axis = 2, beam_sign = 1;
    long long nvox = 0;
    int device = 0;
    int16_t *hu = nullptr;
    float *rho = nullptr;
    float2 *mat = nullptr;                   // (rho, SPR) per voxel, built on first use
    std::mutex mat_mutex;
    std::atomic<int> refs{1};
};

struct PhaseState {
    unsigned long long *tally = nullptr;
    float *dose = nullptr;
    unsigned long long *ledger = nullptr;
    unsigned long long *prefix = nullptr;
    float *wh = nullptr;
    unsigned long long *rem = nullptr;
    uint64_t n_hist = 0;
    bool allocated = false;     // histories allocated for n_hist
    bool has_dose = false;
};

}  // namespace

struct dose_ctx {
    Grid *g = nullptr;
    int n_spots = 0;
    float4 *spot = nullptr;
    unsigned long long *protons = nullptr;
    int *layer = nullptr;
    int *field = nullptr;
    unsigned long long *pp = nullptr;
    int n_fields = 0;
    int *start_phase = nullptr;
    long long *field_end = nullptr;
    bool have_plan = false;
    bool have_delivery = false;              // the plan ran through the timeline
    signed char field_dir[64];               // per field: 2 axis + (sign > 0), -1 = the grid's beam
    unsigned char *spot_dir = nullptr;       // per spot beam code, null when every field uses the grid's
    TimelineArgs *tl_args = nullptr;         // device timeline arguments, cap_tl entries
    int cap_tl = 0;
    dose_delivery_spread *tl_spread = nullptr;
    dose_delivery *tl_used = nullptr;        // the delivery the timeline ran
    int *tl_status = nullptr;
    std::vector<PhaseState> ph;
    unsigned long long *tally_all = nullptr; // n_phases x nvox
    float *dose_all = nullptr;               // n_phases x nvox
    unsigned long long *ledger_all = nullptr;// n_phases x LED_WORDS
    unsigned long long *em = nullptr;        // E then M, n_phases x nvox each
    float *dvf_buf = nullptr;                // staging for host DVFs
    float4 *dvf4 = nullptr;                  // one phase's field, interleaved (EMTM)
    unsigned *reach = nullptr;               // n_phases x kReachWords (accumulations)
    uint8_t *mask_buf = nullptr;             // staging for a host mask
    float *dvfgrid_e = nullptr;              // decoded registration grid (r_f - r0), 3 x cap
    float *dvfgrid_delta = nullptr;          // staging for host translations, 3 x cap
    size_t dvfgrid_cap = 0;                  // grid voxels the two buffers hold
    unsigned *maxbits = nullptr;
    unsigned long long *emtm_stats = nullptr;
    float *accum = nullptr;
    bool have_accum = false;
    int accum_method = 0;              // method of the last accumulation
    TJob *d_jobs = nullptr;
    int cap_jobs = 0;
    AllocJob *d_alloc = nullptr;
    NormJob *d_norm = nullptr;
    int cap_aux = 0;
    unsigned long long *d_counter = nullptr;
    unsigned physics = DOSE_PHYS_ALL;
    unsigned max_steps = 20000;
    int block = 1024;                        // launch-shape defaults: the shape the autotuner
    int blocks_per_sm = 0;                   // picks for most workloads (64 registers, 32 warps
    unsigned chunk = 32;                     // per SM)
    int regs = 1;
    int material_grid = 0;                   // DOSE_OPT_MATERIAL_GRID
    long long timeout_ms = 600000;
    long long fail_alloc_after = -1;
    std::vector<std::pair<void *, size_t>> owned;   // device blocks and their sizes
    std::string err;
};

namespace {

int fail(dose_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_thread_err = buf;
    return code;
}

#define CK(c, call)                                                                      \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail((c), DOSE_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
    } while (0)

cudaStream_t S(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Device blocks released by destroyed contexts, kept per (device, size) for
// the next context (cudaMalloc/cudaFree cost ~0.1 ms each and cudaFree
// synchronises the device).  Blocks enter the cache only after
// dose_destroy has synchronised the device, so no kernel still uses them;
// at most kBlockCacheBytes are kept, and an allocation that fails empties
// the cache and tries again.
std::mutex g_cache_mutex;
std::map<std::pair<int, size_t>, std::vector<void *>> g_cache;
size_t g_cache_bytes = 0;
constexpr size_t kBlockCacheBytes = size_t(8) << 30;

size_t block_size(size_t bytes) { return (std::max<size_t>(bytes, 16) + 255) & ~size_t(255); }

void cache_flush(int dev)
{
    std::lock_guard<std::mutex> lock(g_cache_mutex);
    for (auto it = g_cache.begin(); it != g_cache.end();) {
        if (it->first.first != dev) { ++it; continue; }
        for (void *q : it->second) { cudaFree(q); g_cache_bytes -= it->first.second; }
        it = g_cache.erase(it);
    }
}

// A device block of block_size(bytes) on the current device.
cudaError_t block_alloc(void **p, size_t bytes)
{
    const size_t sz = block_size(bytes);
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        auto it = g_cache.find({dev, sz});
        if (it != g_cache.end() && !it->second.empty()) {
            *p = it->second.back();
            it->second.pop_back();
            g_cache_bytes -= sz;
            return cudaSuccess;
        }
    }
    cudaError_t e = cudaMalloc(p, sz);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        cache_flush(dev);
        e = cudaMalloc(p, sz);
    }
    return e;
}

// Give back a block no kernel uses any more (the device was synchronised).
void block_release(void *p, size_t bytes)
{
    if (!p) return;
    const size_t sz = block_size(bytes);
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(g_cache_mutex);
        if (g_cache_bytes + sz <= kBlockCacheBytes) {
            g_cache[{dev, sz}].push_back(p);
            g_cache_bytes += sz;
            return;
        }
    }
    cudaFree(p);
}

int dalloc(dose_ctx *c, void **p, size_t bytes)
{
    if (c->fail_alloc_after >= 0) {
        if (c->fail_alloc_after == 0) {
            *p = nullptr;
            return fail(c, DOSE_ENOMEM, "device allocation of %zu bytes failed (injected)", bytes);
        }
        --c->fail_alloc_after;
    }
    cudaError_t e = block_alloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, DOSE_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->owned.emplace_back(*p, bytes);
    return DOSE_OK;
}

// Free one block while the context lives: cudaFree (it waits for the device).
void dfree(dose_ctx *c, void *p)
{
    if (!p) return;
    auto it = std::find_if(c->owned.begin(), c->owned.end(), [p](const std::pair<void *, size_t> &o) { return o.first == p; });
    if (it != c->owned.end()) c->owned.erase(it);
    cudaFree(p);
}

template <class T>
int dalloc_t(dose_ctx *c, T **p, size_t count)
{
    return dalloc(c, reinterpret_cast<void **>(p), count * sizeof(T));
}

int device_tables(dose_ctx *c, int dev, DeviceTables *out)
{
    std::lock_guard<std::mutex> lock(g_tab_mutex);
    if (dev < 0 || dev >= kMaxDevices) return fail(c, DOSE_ECUDA, "device %d out of range", dev);
    if (!g_host_tables) {
        g_host_tables = new Tables;
        build_tables(g_host_tables, &g_host_inv_ds);
    }
    if (!g_tab[dev].dev) {
        Tables *t = nullptr;
        cudaError_t e = cudaMalloc(&t, sizeof(Tables));
        if (e != cudaSuccess) return fail(c, DOSE_ENOMEM, "tables: %s", cudaGetErrorString(e));
        e = cudaMemcpy(t, g_host_tables, sizeof(Tables), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(t); return fail(c, DOSE_ECUDA, "tables: %s", cudaGetErrorString(e)); }
        g_tab[dev].dev = t;
        g_tab[dev].inv_ds = g_host_inv_ds;
    }
    *out = g_tab[dev];
    return DOSE_OK;
}

int use_device(dose_ctx *c)
{
    CK(c, cudaSetDevice(c->g->device));
    return DOSE_OK;
}

// Tallies, doses and ledgers of all phases live in three contiguous arrays
// (phase-major), allocated on first use.
int ensure_results(dose_ctx *c, cudaStream_t st)
{
    if (c->tally_all) return DOSE_OK;
    const size_t nvox = (size_t)c->g->nvox, P = (size_t)c->g->n_phases;
    int rc;
    if ((rc = dalloc_t(c, &c->tally_all, P * nvox)) || (rc = dalloc_t(c, &c->dose_all, P * nvox)) ||
        (rc = dalloc_t(c, &c->ledger_all, P * LED_WORDS))) {
        dfree(c, c->tally_all); dfree(c, c->dose_all); dfree(c, c->ledger_all);
        c->tally_all = nullptr; c->dose_all = nullptr; c->ledger_all = nullptr;
        return rc;
    }
    CK(c, cudaMemsetAsync(c->ledger_all, 0, P * LED_WORDS * sizeof(unsigned long long), st));
    for (size_t p = 0; p < P; ++p) {
        c->ph[p].tally = c->tally_all + p * nvox;
        c->ph[p].dose = c->dose_all + p * nvox;
        c->ph[p].ledger = c->ledger_all + p * LED_WORDS;
    }
    return DOSE_OK;
}

int ensure_phase(dose_ctx *c, int p, cudaStream_t st)
{
    int rc;
    if ((rc = ensure_results(c, st))) return rc;
    PhaseState &P = c->ph[p];
    if (!P.prefix) {
        const int S = std::max(c->n_spots, 1);
        if ((rc = dalloc_t(c, &P.prefix, S + 1))) return rc;
        if ((rc = dalloc_t(c, &P.wh, S))) return rc;
        if ((rc = dalloc_t(c, &P.rem, S))) return rc;
    }
    return DOSE_OK;
}

int ensure_workspace(dose_ctx *c, int n_jobs)
{
    int rc;
    if (!c->d_counter && (rc = dalloc_t(c, &c->d_counter, 2))) return rc;
    if (n_jobs > c->cap_jobs) {
        dfree(c, c->d_jobs); dfree(c, c->d_alloc); dfree(c, c->d_norm);
        c->d_jobs = nullptr; c->d_alloc = nullptr; c->d_norm = nullptr;
        const int cap = std::max(n_jobs, 16);
        if ((rc = dalloc_t(c, &c->d_jobs, cap))) return rc;
        if ((rc = dalloc_t(c, &c->d_alloc, cap))) return rc;
        if ((rc = dalloc_t(c, &c->d_norm, cap))) return rc;
        c->cap_jobs = c->cap_aux = cap;
    }
    return DOSE_OK;
}

void free_plan(dose_ctx *c)
{
    dfree(c, c->spot); dfree(c, c->protons); dfree(c, c->layer); dfree(c, c->field);
    dfree(c, c->pp); dfree(c, c->start_phase); dfree(c, c->field_end); dfree(c, c->spot_dir);
    c->spot_dir = nullptr;
    c->spot = nullptr; c->protons = nullptr; c->layer = nullptr; c->field = nullptr;
    c->pp = nullptr; c->start_phase = nullptr; c->field_end = nullptr;
    for (auto &P : c->ph) {
        dfree(c, P.prefix); dfree(c, P.wh); dfree(c, P.rem);
        P.prefix = nullptr; P.wh = nullptr; P.rem = nullptr;
        P.allocated = false; P.has_dose = false; P.n_hist = 0;
    }
    c->have_plan = false;
    c->have_delivery = false;
    c->have_accum = false;
    c->n_spots = 0;
}

// Wait for `ev` with a bound; DOSE_ETIMEOUT if it does not complete.
int wait_event(dose_ctx *c, cudaEvent_t ev)
{
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return DOSE_OK;
        if (e != cudaErrorNotReady) return fail(c, DOSE_ECUDA, "wait: %s", cudaGetErrorString(e));
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
            std::chrono::steady_clock::now() - t0).count();
        if (ms > c->timeout_ms) return fail(c, DOSE_ETIMEOUT, "device work did not finish within %lld ms", c->timeout_ms);
        // short naps while the work is young (a dose run of ~10 ms should be
        // noticed within tens of microseconds), longer ones for long runs
        std::this_thread::sleep_for(std::chrono::microseconds(ms < 50 ? 10 : ms < 1000 ? 100 : 1000));
    }
}

int sync_stream(dose_ctx *c, cudaStream_t st)
{
    cudaEvent_t ev;
    CK(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, st);
    int rc = e == cudaSuccess ? wait_event(c, ev) : fail(c, DOSE_ECUDA, "record: %s", cudaGetErrorString(e));
    cudaEventDestroy(ev);
    return rc;
}

bool finite3(const float *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

}  // namespace

namespace dose {
void set_thread_error(const char *msg) { g_thread_err = msg; }

void grid_info(const dose_ctx *c, int dims[4])
{
    dims[0] = c->g->n[0]; dims[1] = c->g->n[1]; dims[2] = c->g->n[2]; dims[3] = c->g->n_phases;
}

int set_phase_zero(dose_ctx *c, int phase, void *stream)
{
    int rc;
    if ((rc = use_device(c))) return rc;
    if ((rc = ensure_results(c, S(stream)))) return rc;
    CK(c, cudaMemsetAsync(c->ph[phase].dose, 0, c->g->nvox * sizeof(float), S(stream)));
    c->ph[phase].has_dose = true;
    c->have_accum = false;
    return DOSE_OK;
}

int copy_plan(dose_ctx *dst, const dose_ctx *src, void *stream)
{
    if (!dst || !src) return fail(dst, DOSE_EINVAL, "contexts are required");
    if (!src->have_plan) return fail(dst, DOSE_ESTATE, "no plan to copy");
    if (dst->g != src->g) return fail(dst, DOSE_EINVAL, "a plan is copied between views of one grid only");
    int rc;
    if ((rc = use_device(dst))) return rc;
    free_plan(dst);
    const size_t n = (size_t)src->n_spots, P = (size_t)src->g->n_phases, F = (size_t)src->n_fields;
    if ((rc = dalloc_t(dst, &dst->spot, n)) || (rc = dalloc_t(dst, &dst->protons, n)) ||
        (rc = dalloc_t(dst, &dst->layer, n)) || (rc = dalloc_t(dst, &dst->field, n)) ||
        (rc = dalloc_t(dst, &dst->pp, n * P)) || (rc = dalloc_t(dst, &dst->start_phase, F)) ||
        (rc = dalloc_t(dst, &dst->field_end, F)) || (src->spot_dir && (rc = dalloc_t(dst, &dst->spot_dir, n)))) {
        free_plan(dst);
        return rc;
    }
    if (!dst->tl_used && ((rc = dalloc_t(dst, &dst->tl_used, 1)) || (rc = dalloc_t(dst, &dst->tl_status, 1)))) return rc;
    cudaStream_t st = S(stream);
    const auto d2d = [&](void *to, const void *from, size_t bytes) {
        return cudaMemcpyAsync(to, from, bytes, cudaMemcpyDeviceToDevice, st);
    };
    CK(dst, d2d(dst->spot, src->spot, n * sizeof(float4)));
    CK(dst, d2d(dst->protons, src->protons, n * sizeof(unsigned long long)));
    CK(dst, d2d(dst->layer, src->layer, n * sizeof(int)));
    CK(dst, d2d(dst->field, src->field, n * sizeof(int)));
    CK(dst, d2d(dst->pp, src->pp, n * P * sizeof(unsigned long long)));
    CK(dst, d2d(dst->start_phase, src->start_phase, F * sizeof(int)));
    CK(dst, d2d(dst->field_end, src->field_end, F * sizeof(long long)));
    if (src->spot_dir) CK(dst, d2d(dst->spot_dir, src->spot_dir, n));
    if (src->have_delivery) CK(dst, d2d(dst->tl_used, src->tl_used, sizeof(dose_delivery)));
    CK(dst, cudaMemsetAsync(dst->tl_status, 0, sizeof(int), st));
    std::memcpy(dst->field_dir, src->field_dir, sizeof dst->field_dir);
    dst->n_spots = src->n_spots;
    dst->n_fields = src->n_fields;
    dst->have_plan = true;
    dst->have_delivery = src->have_delivery;
    return DOSE_OK;
}
}  // namespace dose

// ======================================================================== ABI
extern "C" {

int dose_version(void) { return kVersion; }

const char *dose_last_error(const dose_ctx *c)
{
    return c ? c->err.c_str() : g_thread_err.c_str();
}

int dose_create_grid(dose_ctx **out, int nx, int ny, int nz, float dx_mm, float dy_mm, float dz_mm,
                     const float origin_mm[3], int n_phases, const int16_t *hu, int hu_on_device,
                     const float beam_dir[3], void *stream)
{
    if (!out) return fail(nullptr, DOSE_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(nullptr, DOSE_EINVAL, "grid dimensions must be positive");
    if ((long long)nx * ny * nz > (1ll << 31) - 1)
        return fail(nullptr, DOSE_EINVAL, "grid of %lld voxels exceeds 2^31-1", (long long)nx * ny * nz);
    if (!(dx_mm > 0 && dy_mm > 0 && dz_mm > 0) || !std::isfinite(dx_mm) || !std::isfinite(dy_mm) || !std::isfinite(dz_mm))
        return fail(nullptr, DOSE_EINVAL, "voxel sizes must be positive and finite");
    if (!origin_mm || !finite3(origin_mm)) return fail(nullptr, DOSE_EINVAL, "origin must be 3 finite values");
    if (n_phases <= 0 || n_phases > 4096) return fail(nullptr, DOSE_EINVAL, "n_phases must be in 1..4096");
    if (!hu) return fail(nullptr, DOSE_EINVAL, "hu is NULL");
    if (!beam_dir) return fail(nullptr, DOSE_EINVAL, "beam_dir is NULL");
    int axis = -1, sign = 0, nz_count = 0;
    for (int k = 0; k < 3; ++k) {
        if (beam_dir[k] == 1.0f || beam_dir[k] == -1.0f) { axis = k; sign = beam_dir[k] > 0 ? 1 : -1; ++nz_count; }
        else if (beam_dir[k] != 0.0f) return fail(nullptr, DOSE_EINVAL, "beam_dir must be a unit axis vector");
    }
    if (nz_count != 1) return fail(nullptr, DOSE_EINVAL, "beam_dir must be a unit axis vector");

    dose_ctx *c = new dose_ctx;
    std::memset(c->field_dir, -1, sizeof c->field_dir);
    c->g = new Grid;
    Grid &g = *c->g;
    g.n[0] = nx; g.n[1] = ny; g.n[2] = nz;
    g.d[0] = dx_mm; g.d[1] = dy_mm; g.d[2] = dz_mm;
    for (int k = 0; k < 3; ++k) g.origin[k] = origin_mm[k];
    g.n_phases = n_phases;
    g.beam_axis = axis; g.beam_sign = sign;
    g.nvox = (long long)nx * ny * nz;
    c->ph.resize(n_phases);
    int rc = DOSE_OK;
    cudaError_t e = cudaGetDevice(&g.device);
    if (e != cudaSuccess) {
        rc = fail(nullptr, DOSE_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
        delete c->g; delete c;
        return rc;
    }
    DeviceTables tab;
    const size_t n_all = (size_t)g.nvox * n_phases;
    if ((rc = device_tables(c, g.device, &tab))) {
        g_thread_err = c->err;
        dose_destroy(c);
        return rc;
    }
    e = block_alloc(reinterpret_cast<void **>(&g.hu), n_all * sizeof(int16_t));
    if (e == cudaSuccess) e = block_alloc(reinterpret_cast<void **>(&g.rho), n_all * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        rc = fail(nullptr, DOSE_ENOMEM, "grid allocation (%zu voxels): %s", n_all, cudaGetErrorString(e));
        dose_destroy(c);
        return rc;
    }
    e = cudaMemcpyAsync(g.hu, hu, n_all * sizeof(int16_t),
                        hu_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S(stream));
    if (e == cudaSuccess) {
        k_density<<<1184, 256, 0, S(stream)>>>(g.hu, g.rho, (long long)n_all, tab.dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        rc = fail(nullptr, DOSE_ECUDA, "grid upload: %s", cudaGetErrorString(e));
        dose_destroy(c);
        return rc;
    }
    *out = c;
    return DOSE_OK;
}

int dose_create_view(dose_ctx *base, dose_ctx **out)
{
    if (!out) return fail(nullptr, DOSE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!base) return fail(nullptr, DOSE_EINVAL, "base is NULL");
    dose_ctx *c = new dose_ctx;
    c->g = base->g;
    c->g->refs.fetch_add(1);
    std::memcpy(c->field_dir, base->field_dir, sizeof c->field_dir);
    c->ph.resize(c->g->n_phases);
    c->physics = base->physics;
    c->max_steps = base->max_steps;
    c->block = base->block;
    c->blocks_per_sm = base->blocks_per_sm;
    c->chunk = base->chunk;
    c->regs = base->regs;
    c->material_grid = base->material_grid;
    c->timeout_ms = base->timeout_ms;
    *out = c;
    return DOSE_OK;
}

int dose_get_option(const dose_ctx *c, int option, int64_t *value)
{
    if (!c || !value) return fail(nullptr, DOSE_EINVAL, "ctx and value are required");
    switch (option) {
    case DOSE_OPT_PHYSICS: *value = c->physics; return DOSE_OK;
    case DOSE_OPT_MAX_STEPS: *value = c->max_steps; return DOSE_OK;
    case DOSE_OPT_BLOCK: *value = c->block; return DOSE_OK;
    case DOSE_OPT_BLOCKS_PER_SM: *value = c->blocks_per_sm; return DOSE_OK;
    case DOSE_OPT_CHUNK: *value = c->chunk; return DOSE_OK;
    case DOSE_OPT_TIMEOUT_MS: *value = c->timeout_ms; return DOSE_OK;
    case DOSE_OPT_FAIL_ALLOC_AFTER: *value = c->fail_alloc_after; return DOSE_OK;
    case DOSE_OPT_REGISTERS: *value = c->regs; return DOSE_OK;
    case DOSE_OPT_MATERIAL_GRID: *value = c->material_grid; return DOSE_OK;
    default: return fail(nullptr, DOSE_EINVAL, "unknown option %d", option);
    }
}

int dose_set_option(dose_ctx *c, int option, int64_t value)
{
    if (!c) return fail(nullptr, DOSE_EINVAL, "ctx is NULL");
    switch (option) {
    case DOSE_OPT_PHYSICS:
        if (value < 0 || value > 7) return fail(c, DOSE_EINVAL, "physics mask must be in 0..7");
        c->physics = (unsigned)value; return DOSE_OK;
    case DOSE_OPT_MAX_STEPS:
        if (value < 1 || value > 100000000) return fail(c, DOSE_EINVAL, "max steps must be in 1..1e8");
        c->max_steps = (unsigned)value; return DOSE_OK;
    case DOSE_OPT_BLOCK:
        if (value < 64 || value > 1024 || value % 32) return fail(c, DOSE_EINVAL, "block must be a multiple of 32 in 64..1024");
        c->block = (int)value; return DOSE_OK;
    case DOSE_OPT_BLOCKS_PER_SM:
        if (value < 0 || value > 32) return fail(c, DOSE_EINVAL, "blocks per SM must be in 0..32");
        c->blocks_per_sm = (int)value; return DOSE_OK;
    case DOSE_OPT_CHUNK:
        if (value < 1 || value > (1 << 20)) return fail(c, DOSE_EINVAL, "chunk must be in 1..2^20");
        c->chunk = (unsigned)value; return DOSE_OK;
    case DOSE_OPT_TIMEOUT_MS:
        if (value < 1) return fail(c, DOSE_EINVAL, "timeout must be positive");
        c->timeout_ms = value; return DOSE_OK;
    case DOSE_OPT_FAIL_ALLOC_AFTER:
        c->fail_alloc_after = value < 0 ? -1 : value; return DOSE_OK;
    case DOSE_OPT_REGISTERS:
        if (value != 0 && value != 1) return fail(c, DOSE_EINVAL, "register option must be 0 or 1");
        c->regs = (int)value; return DOSE_OK;
    case DOSE_OPT_MATERIAL_GRID:
        if (value != 0 && value != 1) return fail(c, DOSE_EINVAL, "material-grid option must be 0 or 1");
        c->material_grid = (int)value; return DOSE_OK;
    default:
        return fail(c, DOSE_EINVAL, "unknown option %d", option);
    }
}

namespace {

// Check a plan's spots; n_fields and the proton total on success.
int check_spots(dose_ctx *c, const dose_spot *spots, int64_t n, int *n_fields, unsigned long long *total)
{
    if (!spots) return fail(c, DOSE_EINVAL, "spots is NULL");
    if (n <= 0 || n > kMaxSpots) return fail(c, DOSE_EINVAL, "number of spots must be in 1..%d", kMaxSpots);
    int nf = 0;
    unsigned long long tot = 0;
    for (int64_t s = 0; s < n; ++s) {
        const dose_spot &q = spots[s];
        if (!(q.energy_MeV >= 1.0f && q.energy_MeV <= 250.0f))
            return fail(c, DOSE_EINVAL, "spot %lld: energy %g MeV outside 1..250", (long long)s, q.energy_MeV);
        if (!(q.sigma_mm >= 0.0f) || !std::isfinite(q.sigma_mm) || !std::isfinite(q.x_mm) || !std::isfinite(q.y_mm))
            return fail(c, DOSE_EINVAL, "spot %lld: position and sigma must be finite, sigma >= 0", (long long)s);
        if (q.field < 0 || q.field >= kMaxFields)
            return fail(c, DOSE_EINVAL, "spot %lld: field %d outside 0..%d", (long long)s, q.field, kMaxFields - 1);
        nf = std::max(nf, q.field + 1);
        if (tot + q.protons < tot) return fail(c, DOSE_EINVAL, "total protons overflow 64 bits");
        tot += q.protons;
    }
    *n_fields = nf;
    *total = tot;
    return DOSE_OK;
}

// A delivery the clock can run: the grid's phase count, the progress
// conditions, and a clock far from overflow.
int check_delivery(dose_ctx *c, const dose_delivery *dl, int64_t n, unsigned long long total)
{
    const int P = c->g->n_phases;
    if (dl->n_phases != P) return fail(c, DOSE_EINVAL, "delivery n_phases %d != grid phases %d", dl->n_phases, P);
    if (!delivery_ok(*dl))
        return fail(c, DOSE_EINVAL, "delivery parameters out of range or unable to progress (period, sigma, "
                                    "gate window, discard, extraction limit, repainting)");
    const long double spill = (long double)total * 1e9L / (long double)dl->rate_protons_per_s;
    const long double paints = dl->max_protons_per_paint ? (long double)total / dl->max_protons_per_paint + 1 : dl->repaints;
    const long double sw = (long double)n * paints * (long double)std::max(dl->spot_switch_ns, dl->layer_switch_ns);
    const long double waits = (long double)n * paints * (long double)(dl->period_ns + 6 * dl->period_sigma_ns);
    if (spill + sw + waits > 4.0e18L) return fail(c, DOSE_EINVAL, "delivery clock would overflow");
    return DOSE_OK;
}

// The grid's per-voxel (rho, SPR), built once on first use (views share it).
int ensure_material(dose_ctx *c, cudaStream_t st)
{
    Grid &g = *c->g;
    std::lock_guard<std::mutex> lock(g.mat_mutex);
    if (g.mat) return DOSE_OK;
    const size_t n_all = (size_t)g.nvox * g.n_phases;
    cudaError_t e = block_alloc(reinterpret_cast<void **>(&g.mat), n_all * sizeof(float2));
    if (e != cudaSuccess) {
        cudaGetLastError();
        g.mat = nullptr;
        return fail(c, DOSE_ENOMEM, "material grid (%zu bytes): %s", n_all * sizeof(float2), cudaGetErrorString(e));
    }
    DeviceTables tab;
    int rc;
    if ((rc = device_tables(c, g.device, &tab))) return rc;
    k_material<<<1184, 256, 0, st>>>(g.hu, g.mat, (long long)n_all, tab.dev);
    CK(c, cudaGetLastError());
    return DOSE_OK;
}

// Per-spot beam codes from the fields' directions (none when every field of
// the plan enters along the grid's beam).
int upload_spot_dirs(dose_ctx *c, const int *field, cudaStream_t st)
{
    bool any = false;
    for (int s = 0; s < c->n_spots; ++s) any |= c->field_dir[field[s]] >= 0;
    dfree(c, c->spot_dir);
    c->spot_dir = nullptr;
    if (!any) return DOSE_OK;
    const unsigned char grid_code = (unsigned char)(2 * c->g->beam_axis + (c->g->beam_sign > 0 ? 1 : 0));
    std::vector<unsigned char> code(c->n_spots);
    for (int s = 0; s < c->n_spots; ++s)
        code[s] = c->field_dir[field[s]] >= 0 ? (unsigned char)c->field_dir[field[s]] : grid_code;
    int rc;
    if ((rc = dalloc_t(c, &c->spot_dir, (size_t)c->n_spots))) return rc;
    // from pageable memory: returns once the bytes are staged
    CK(c, cudaMemcpyAsync(c->spot_dir, code.data(), code.size(), cudaMemcpyHostToDevice, st));
    return DOSE_OK;
}

// Replace the plan of c and upload the spots.
int load_plan(dose_ctx *c, const dose_spot *spots, int64_t n, int n_fields, cudaStream_t st)
{
    int rc;
    if ((rc = use_device(c))) return rc;
    free_plan(c);
    const int P = c->g->n_phases;
    std::vector<float4> sp(n);
    std::vector<unsigned long long> pr(n);
    std::vector<int> la(n), fi(n);
    for (int64_t s = 0; s < n; ++s) {
        sp[s] = make_float4(spots[s].x_mm, spots[s].y_mm, spots[s].energy_MeV, spots[s].sigma_mm);
        pr[s] = spots[s].protons;
        la[s] = spots[s].layer;
        fi[s] = spots[s].field;
    }
    c->n_spots = (int)n;
    c->n_fields = n_fields;
    if ((rc = dalloc_t(c, &c->spot, n)) || (rc = dalloc_t(c, &c->protons, n)) ||
        (rc = dalloc_t(c, &c->layer, n)) || (rc = dalloc_t(c, &c->field, n)) ||
        (rc = dalloc_t(c, &c->pp, (size_t)n * P)) || (rc = dalloc_t(c, &c->start_phase, n_fields)) ||
        (rc = dalloc_t(c, &c->field_end, n_fields))) {
        free_plan(c);
        return rc;
    }
    if (!c->tl_used && ((rc = dalloc_t(c, &c->tl_used, 1)) || (rc = dalloc_t(c, &c->tl_status, 1)))) return rc;
    CK(c, cudaMemcpyAsync(c->spot, sp.data(), n * sizeof(float4), cudaMemcpyHostToDevice, st));
    CK(c, cudaMemcpyAsync(c->protons, pr.data(), n * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
    CK(c, cudaMemcpyAsync(c->layer, la.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(c, cudaMemcpyAsync(c->field, fi.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(c, cudaMemsetAsync(c->pp, 0, (size_t)n * P * sizeof(unsigned long long), st));
    CK(c, cudaMemsetAsync(c->tl_status, 0, sizeof(int), st));
    return upload_spot_dirs(c, fi.data(), st);
}

TimelineArgs timeline_args(dose_ctx *c, const dose_delivery &d)
{
    TimelineArgs a;
    a.protons = c->protons; a.layer = c->layer; a.field = c->field;
    a.n_spots = c->n_spots; a.n_fields = c->n_fields;
    a.d = d; a.spread = nullptr; a.trial = 0;
    a.pp = c->pp; a.field_end = c->field_end; a.start_out = c->start_phase;
    a.used = c->tl_used; a.status = c->tl_status;
    return a;
}

// Launch the timelines of `args` (one block each) from c's argument buffer.
int launch_timelines(dose_ctx *c, const std::vector<TimelineArgs> &args, cudaStream_t st)
{
    int rc;
    if ((int)args.size() > c->cap_tl) {
        if (c->tl_args) { dfree(c, c->tl_args); c->tl_args = nullptr; c->cap_tl = 0; }
        if ((rc = dalloc_t(c, &c->tl_args, args.size()))) return rc;
        c->cap_tl = (int)args.size();
    }
    CK(c, cudaMemcpyAsync(c->tl_args, args.data(), args.size() * sizeof(TimelineArgs), cudaMemcpyHostToDevice, st));
    // the plan's protons, layers and fields are staged in shared memory
    const size_t smem = (size_t)args[0].n_spots * (sizeof(unsigned long long) + sizeof(int) + 1);
    if (smem > 48 * 1024)
        CK(c, cudaFuncSetAttribute(k_timeline, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_timeline<<<(unsigned)args.size(), kMaxFields, smem, st>>>(c->tl_args);
    CK(c, cudaGetLastError());
    return DOSE_OK;
}

// Wait for the stream and turn a timeline status into an error.
int timeline_status(dose_ctx *c, dose_ctx *report, int trial, bool is_trial, cudaStream_t st)
{
    int rc, status = 0;
    if ((rc = sync_stream(report, st))) return rc;
    CK(report, cudaMemcpy(&status, c->tl_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status == 0) return DOSE_OK;
    c->have_plan = false;
    const char *why = status == 1 ? "sampled delivery breaks the progress conditions"
                    : status == 2 ? "delivery makes no progress (fills deliver nothing)"
                                  : "delivery clock overflow";
    if (is_trial) return fail(report, DOSE_EINVAL, "trial %d: %s", trial, why);
    return fail(report, DOSE_EINVAL, "%s", why);
}

}  // namespace

int dose_set_field_beam(dose_ctx *c, int field, const float beam_dir[3])
{
    if (!c) return fail(nullptr, DOSE_EINVAL, "ctx is NULL");
    if (field < 0 || field >= kMaxFields) return fail(c, DOSE_EINVAL, "field %d outside 0..%d", field, kMaxFields - 1);
    signed char code = -1;
    if (beam_dir) {
        int axis = -1, n = 0, sign = 1;
        for (int k = 0; k < 3; ++k) {
            if (beam_dir[k] == 1.0f || beam_dir[k] == -1.0f) { axis = k; sign = beam_dir[k] > 0 ? 1 : -1; ++n; }
            else if (beam_dir[k] != 0.0f) return fail(c, DOSE_EINVAL, "beam_dir must be a unit axis vector");
        }
        if (n != 1) return fail(c, DOSE_EINVAL, "beam_dir must be a unit axis vector");
        code = (signed char)(2 * axis + (sign > 0 ? 1 : 0));
    }
    c->field_dir[field] = code;
    if (!c->have_plan) return DOSE_OK;
    // re-derive the loaded plan's spot codes
    std::vector<int> fi(c->n_spots);
    int rc;
    if ((rc = use_device(c))) return rc;
    CK(c, cudaMemcpy(fi.data(), c->field, fi.size() * sizeof(int), cudaMemcpyDeviceToHost));
    return upload_spot_dirs(c, fi.data(), nullptr);
}

int dose_add_spots(dose_ctx *c, const dose_spot *spots, int64_t n, const dose_delivery *dl, void *stream)
{
    if (!c) return fail(nullptr, DOSE_EINVAL, "ctx is NULL");
    int n_fields = 0, rc;
    unsigned long long total = 0;
    if ((rc = check_spots(c, spots, n, &n_fields, &total))) return rc;
    if (dl && (rc = check_delivery(c, dl, n, total))) return rc;
    cudaStream_t st = S(stream);
    if ((rc = load_plan(c, spots, n, n_fields, st))) return rc;
    if (dl) {
        if ((rc = launch_timelines(c, {timeline_args(c, *dl)}, st))) return rc;
        c->have_plan = true;
        c->have_delivery = true;
        if (dl->synchrotron && (rc = timeline_status(c, c, 0, false, st))) return rc;
    } else {
        CK(c, cudaMemcpyAsync(c->pp, c->protons, n * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st));
        CK(c, cudaMemsetAsync(c->start_phase, 0, n_fields * sizeof(int), st));
        CK(c, cudaMemsetAsync(c->field_end, 0, n_fields * sizeof(long long), st));
        c->have_plan = true;
    }
    return DOSE_OK;
}

int dose_add_spots_trials(dose_ctx *const *ctxs, int n_trials, const dose_spot *spots, int64_t n,
                          const dose_delivery *mean, const dose_delivery_spread *spread, uint64_t first_trial,
                          void *stream)
{
    if (!ctxs || n_trials <= 0 || !ctxs[0]) return fail(nullptr, DOSE_EINVAL, "no contexts");
    dose_ctx *c0 = ctxs[0];
    if (!mean || !spread) return fail(c0, DOSE_EINVAL, "mean delivery and spread are required");
    for (int k = 0; k < n_trials; ++k) {
        if (!ctxs[k]) return fail(c0, DOSE_EINVAL, "context %d is NULL", k);
        if (ctxs[k]->g->device != c0->g->device) return fail(c0, DOSE_EINVAL, "context %d is on another GPU", k);
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == ctxs[k]) return fail(c0, DOSE_EINVAL, "context %d appears twice", k);
    }
    const dose_delivery_spread &sp = *spread;
    const int64_t sig[6] = {sp.spot_switch_sigma_ns, sp.layer_switch_sigma_ns, sp.discard_sigma_ns,
                            sp.rate_sigma, sp.fill_protons_sigma, sp.extraction_limit_sigma_ns};
    for (int64_t v : sig)
        if (v < 0 || v > (1ll << 38)) return fail(c0, DOSE_EINVAL, "spread sigmas must be in 0..2^38");
    if (sp.period_max_ns > sp.period_min_ns && (sp.period_step_ns <= 0 || sp.period_min_ns <= 0))
        return fail(c0, DOSE_EINVAL, "period range needs a positive minimum and step");
    int n_fields = 0, rc;
    unsigned long long total = 0;
    if ((rc = check_spots(c0, spots, n, &n_fields, &total))) return rc;
    // the mean must be sound; sampled trials are checked in the kernel
    dose_delivery worst = *mean;
    if (sp.period_max_ns > sp.period_min_ns) worst.period_ns = sp.period_min_ns;
    if ((rc = check_delivery(c0, &worst, n, total))) return rc;
    cudaStream_t st = S(stream);
    std::vector<TimelineArgs> args;
    for (int k = 0; k < n_trials; ++k) {
        dose_ctx *c = ctxs[k];
        if (c->g->n_phases != c0->g->n_phases) return fail(c0, DOSE_EINVAL, "context %d has another phase count", k);
        if ((rc = load_plan(c, spots, n, n_fields, st))) return rc;
        args.push_back(timeline_args(c, *mean));
    }
    if (!c0->tl_spread && (rc = dalloc_t(c0, &c0->tl_spread, 1))) return rc;
    CK(c0, cudaMemcpyAsync(c0->tl_spread, spread, sizeof(dose_delivery_spread), cudaMemcpyHostToDevice, st));
    for (int k = 0; k < n_trials; ++k) {
        args[k].spread = c0->tl_spread;
        args[k].trial = first_trial + (uint64_t)k;
    }
    if ((rc = launch_timelines(c0, args, st))) return rc;
    for (int k = 0; k < n_trials; ++k) {
        ctxs[k]->have_plan = true;
        ctxs[k]->have_delivery = true;
    }
    for (int k = 0; k < n_trials; ++k)
        if ((rc = timeline_status(ctxs[k], c0, (int)(first_trial + k), true, st))) return rc;
    return DOSE_OK;
}

int dose_run_batch(const dose_job *jobs, int n_jobs, void *stream)
{
    if (!jobs || n_jobs <= 0) return fail(nullptr, DOSE_EINVAL, "no jobs");
    dose_ctx *c0 = jobs[0].ctx;
    if (!c0) return fail(nullptr, DOSE_EINVAL, "job 0 has no context");
    for (int j = 0; j < n_jobs; ++j) {
        const dose_job &J = jobs[j];
        dose_ctx *c = J.ctx;
        if (!c) return fail(c0, DOSE_EINVAL, "job %d has no context", j);
        if (c->g->device != c0->g->device) return fail(c0, DOSE_EINVAL, "job %d is on another GPU", j);
        if (!c->have_plan) return fail(c0, DOSE_ESTATE, "job %d: no spots loaded", j);
        if (J.phase < 0 || J.phase >= c->g->n_phases) return fail(c0, DOSE_EINVAL, "job %d: phase %d out of range", j, J.phase);
        if (J.n_histories == 0) return fail(c0, DOSE_EINVAL, "job %d: n_histories is 0", j);
        if (J.hist_begin > J.hist_end || J.hist_end > J.n_histories)
            return fail(c0, DOSE_EINVAL, "job %d: history range [%llu, %llu) outside [0, %llu)", j,
                        (unsigned long long)J.hist_begin, (unsigned long long)J.hist_end,
                        (unsigned long long)J.n_histories);
        if (!(J.spr_scale > 0.1f && J.spr_scale < 10.0f)) return fail(c0, DOSE_EINVAL, "job %d: spr_scale out of range", j);
        if (!finite3(J.shift_mm)) return fail(c0, DOSE_EINVAL, "job %d: shift must be finite", j);
        const PhaseState &P = c->ph[J.phase];
        if (!(J.flags & DOSE_JOB_CLEAR) && (!P.allocated || P.n_hist != J.n_histories))
            return fail(c0, DOSE_ESTATE, "job %d: phase not started with DOSE_JOB_CLEAR for %llu histories", j,
                        (unsigned long long)J.n_histories);
        for (int k = 0; k < j; ++k)
            if (jobs[k].ctx == c && jobs[k].phase == J.phase && ((J.flags | jobs[k].flags) & DOSE_JOB_CLEAR))
                return fail(c0, DOSE_EINVAL, "jobs %d and %d clear the same phase", k, j);
    }
    int rc;
    if ((rc = use_device(c0))) return rc;
    DeviceTables tab;
    if ((rc = device_tables(c0, c0->g->device, &tab))) return rc;
    if ((rc = ensure_workspace(c0, n_jobs))) return rc;
    cudaStream_t st = S(stream);
    std::vector<AllocJob> aj;
    std::vector<TJob> tj;
    std::vector<NormJob> nj;
    unsigned long long work = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const dose_job &J = jobs[j];
        dose_ctx *c = J.ctx;
        if ((rc = ensure_phase(c, J.phase, st))) { if (c != c0) c0->err = c->err; return rc; }
        PhaseState &P = c->ph[J.phase];
        const Grid &g = *c->g;
        if (J.flags & DOSE_JOB_CLEAR) {
            CK(c0, cudaMemsetAsync(P.tally, 0, g.nvox * sizeof(unsigned long long), st));
            CK(c0, cudaMemsetAsync(P.ledger, 0, LED_WORDS * sizeof(unsigned long long), st));
            AllocJob a;
            a.protons = c->pp + (size_t)J.phase * c->n_spots;
            a.spot = c->spot;
            a.rem = P.rem; a.prefix = P.prefix; a.wh = P.wh; a.ledger = P.ledger;
            a.n_spots = c->n_spots; a.n_hist = J.n_histories;
            aj.push_back(a);
            P.n_hist = J.n_histories;
            P.allocated = true;
            P.has_dose = false;
            c->have_accum = false;
        }
        const unsigned long long cnt = J.hist_end - J.hist_begin;
        if (cnt) {
            TJob t;
            t.hu = g.hu + (size_t)J.phase * g.nvox;
            t.matg = nullptr;
            if (c0->material_grid) {
                if ((rc = ensure_material(c, st))) { if (c != c0) c0->err = c->err; return rc; }
                t.matg = g.mat + (size_t)J.phase * g.nvox;
            }
            t.tally = P.tally; t.ledger = P.ledger;
            t.spot = c->spot; t.wh = P.wh; t.prefix = P.prefix; t.n_spots = c->n_spots;
            t.nx = g.n[0]; t.ny = g.n[1]; t.nz = g.n[2];
            t.dx = g.d[0]; t.dy = g.d[1]; t.dz = g.d[2];
            t.idx = 1.0f / g.d[0]; t.idy = 1.0f / g.d[1]; t.idz = 1.0f / g.d[2];
            for (int k = 0; k < 3; ++k) t.o[k] = g.origin[k] + J.shift_mm[k];
            t.spot_dir = c->spot_dir;
            t.beam_axis = g.beam_axis; t.beam_sign = g.beam_sign;
            t.spr_scale = J.spr_scale; t.physics = c->physics; t.max_steps = c->max_steps;
            t.key0 = (unsigned)J.seed; t.key1 = (unsigned)(J.seed >> 32);
            for (int r = 0; r < 10; r += 2)   // Philox round keys: key + r x the Weyl increments
                t.rk[r >> 1] = make_uint4(t.key0 + (unsigned)r * 0x9E3779B9u, t.key1 + (unsigned)r * 0xBB67AE85u,
                                          t.key0 + (unsigned)(r + 1) * 0x9E3779B9u, t.key1 + (unsigned)(r + 1) * 0xBB67AE85u);
            t.stream = (unsigned)J.phase;
            t.hist_begin = J.hist_begin; t.work_begin = work; t.n_work = cnt; t.spread_log2 = spread_for(g.nvox, cnt);
            tj.push_back(t);
            work += cnt;
        }
        if (J.flags & DOSE_JOB_FINISH) {
            // the deposited total is re-taken from the tally at each finish
            CK(c0, cudaMemsetAsync(P.ledger + LED_DEP, 0, sizeof(unsigned long long), st));
            NormJob nm;
            nm.tally = P.tally; nm.ledger = P.ledger; nm.rho = g.rho + (size_t)J.phase * g.nvox;
            nm.dose = P.dose; nm.n_hist = J.n_histories;
            nm.voxel_cm3 = (double)g.d[0] * g.d[1] * g.d[2] / 1000.0;
            nm.nvox = g.nvox;
            nj.push_back(nm);
            P.has_dose = true;
        }
    }
    if (!aj.empty()) {
        CK(c0, cudaMemcpyAsync(c0->d_alloc, aj.data(), aj.size() * sizeof(AllocJob), cudaMemcpyHostToDevice, st));
        k_alloc<<<(unsigned)aj.size(), 1024, 0, st>>>(c0->d_alloc);
        CK(c0, cudaGetLastError());
    }
    if (work) {
        if (!c0->regs && c0->block > 512)
            return fail(c0, DOSE_EINVAL, "block %d needs the 64-register variant (DOSE_OPT_REGISTERS 1)", c0->block);
        CK(c0, transport_allow_smem());
        int sms = 0;
        CK(c0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c0->g->device));
        // One launch over a group of jobs whose work items are numbered
        // contiguously from 0.  One job: its descriptor goes in the launch's
        // parameters; several: a table in device memory; a table whose jobs
        // share their per-step fields (the phases of one plan and seed) reads
        // those from the launch's parameters too.
        auto launch_group = [&](const std::vector<TJob> &grp, unsigned long long gwork) -> int {
            const bool single = grp.size() == 1;
            const bool shared = !single && jobs_share_step_fields(grp.data(), (int)grp.size());
            if (!single)
                CK(c0, cudaMemcpyAsync(c0->d_jobs, grp.data(), grp.size() * sizeof(TJob), cudaMemcpyHostToDevice, st));
            CK(c0, cudaMemsetAsync(c0->d_counter, 0, sizeof(unsigned long long), st));
            // a table whose jobs differ only in seed and SPR scale (views of
            // one grid: trials, serving steps) reads the rest from there too
            const bool geom = !single && !shared && jobs_share_geometry(grp.data(), (int)grp.size());
            const int mode = single ? kLaunchSingle : shared ? kLaunchShared : geom ? kLaunchGeom : kLaunchTable;
            const int spec = transport_spec(grp.data(), (int)grp.size());
            const void *kern = transport_kernel(mode, c0->regs, spec);
            size_t smem;
            int stage = 0, fit = 0;
            if (single) {
                smem = transport_smem(1) + birth_smem(c0->block);
                CK(c0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kern, c0->block, smem));
            } else {
                // stage the job table in shared memory unless that costs
                // resident blocks or leaves too little L1 (kStageSmemCap)
                const int n = (int)grp.size();
                const size_t smem_plain = transport_smem(kMaxStagedJobs + 1) + birth_smem(c0->block);
                int fit_plain = 0, fit_staged = 0;
                CK(c0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit_plain, kern, c0->block, smem_plain));
                if (n <= kMaxStagedJobs)
                    CK(c0, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit_staged, kern, c0->block,
                                                                         transport_smem(n) + birth_smem(c0->block)));
                stage = fit_staged > 0 && fit_staged >= fit_plain &&
                        transport_smem(n) + birth_smem(c0->block) <= kStageSmemCap ? 1 : 0;
                smem = stage ? transport_smem(n) + birth_smem(c0->block) : smem_plain;
                fit = stage ? fit_staged : fit_plain;
            }
            int per_sm = c0->blocks_per_sm;
            if (per_sm <= 0) per_sm = fit;
            if (per_sm <= 0) return fail(c0, DOSE_ECUDA, "transport kernel does not fit with block %d", c0->block);
            const unsigned long long warps = (unsigned long long)sms * per_sm * (c0->block / 32);
            // keep at least ~4 pulls per warp so the tail stays short
            unsigned chunk = c0->chunk;
            while (chunk > 32 && (unsigned long long)chunk * warps * 4 > gwork) chunk >>= 1;
            TransportLaunch L;
            L.mode = mode; L.regs = c0->regs; L.spec = spec;
            L.grid = (unsigned)(sms * per_sm); L.block = (unsigned)c0->block; L.smem = smem; L.stream = st;
            L.job0 = grp.data(); L.d_jobs = c0->d_jobs; L.n_jobs = (int)grp.size();
            L.total = gwork; L.counter = c0->d_counter; L.tab = tab.dev; L.inv_ds = tab.inv_ds;
            L.chunk = chunk; L.stage = stage;
            CK(c0, transport_launch(L));
            return DOSE_OK;
        };
        // Jobs that each keep the GPU busy for tens of milliseconds or more
        // (kSplitWork work items) run one after another as single-job
        // launches, the cheapest step; the others share one launch, where
        // the per-launch tail is paid once.
        std::vector<TJob> rest, big;
        unsigned long long rest_work = 0;
        for (const TJob &t0 : tj) {
            TJob t = t0;
            if (tj.size() > 1 && t.n_work >= kSplitWork) {
                t.work_begin = 0;
                big.push_back(t);
            } else {
                t.work_begin = rest_work;
                rest_work += t.n_work;
                rest.push_back(t);
            }
        }
        if (!rest.empty() && (rc = launch_group(rest, rest_work))) return rc;
        for (const TJob &t : big)
            if ((rc = launch_group(std::vector<TJob>{t}, t.n_work))) return rc;
    }
    if (!nj.empty()) {
        CK(c0, cudaMemcpyAsync(c0->d_norm, nj.data(), nj.size() * sizeof(NormJob), cudaMemcpyHostToDevice, st));
        dim3 grid(608, (unsigned)nj.size());
        k_normalise<<<grid, 256, 0, st>>>(c0->d_norm);
        CK(c0, cudaGetLastError());
    }
    return DOSE_OK;
}

int dose_run_phase(dose_ctx *c, int phase, uint64_t n_histories, uint64_t seed, float spr_scale,
                   const float shift_mm[3], void *stream)
{
    if (!c) return fail(nullptr, DOSE_EINVAL, "ctx is NULL");
    dose_job j;
    j.ctx = c; j.phase = phase; j.flags = DOSE_JOB_CLEAR | DOSE_JOB_FINISH;
    j.n_histories = n_histories; j.hist_begin = 0; j.hist_end = n_histories;
    j.seed = seed; j.spr_scale = spr_scale;
    for (int k = 0; k < 3; ++k) j.shift_mm[k] = shift_mm ? shift_mm[k] : 0.0f;
    const int rc = dose_run_batch(&j, 1, stream);
    if (rc && c->err.empty()) c->err = g_thread_err;
    return rc;
}

}  // extern "C"

namespace {

// Time run() (one transport launch of a history sample on `st`) under each
// launch shape -- register variant x block x chunk, then the material source
// for the fastest -- with c's options, which the launches read; leaves the
// winners in c's options (or the previous ones on error).
template <class Run>
int tune_shapes(dose_ctx *c, cudaStream_t st, bool single, Run run, int64_t best[4])
{
    static const int blocks[] = {128, 256, 512, 1024};
    static const unsigned chunks[] = {32, 64, 128, 256};
    const int keep_block = c->block, keep_regs = c->regs, keep_per_sm = c->blocks_per_sm;
    const int keep_mat = c->material_grid;
    const unsigned keep_chunk = c->chunk;
    int best_mat = keep_mat;
    cudaEvent_t e0, e1;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    float best_ms = -1.0f;
    int best_block = keep_block, best_regs = keep_regs;
    unsigned best_chunk = keep_chunk;
    int rc = DOSE_OK;
    auto timed = [&](float *ms) -> int {
        cudaEventRecord(e0, st);
        int r = run();
        if (r) return r;
        cudaEventRecord(e1, st);
        if ((r = sync_stream(c, st))) return r;
        cudaEventElapsedTime(ms, e0, e1);
        return DOSE_OK;
    };
    c->blocks_per_sm = 0;
    // the occupancy query needs the kernels' dynamic shared-memory limit set
    if (transport_allow_smem() != cudaSuccess) { rc = fail(c, DOSE_ECUDA, "cudaFuncSetAttribute failed"); goto done; }
    for (int regs = 0; regs < 2; ++regs) {
        for (int b : blocks) {
            if (!regs && b > 512) continue;
            int fits = 0;
            const void *k = transport_kernel(single ? kLaunchSingle : kLaunchTable, regs, kSpecGeneric);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fits, k, b, transport_smem(1) + birth_smem(b)) != cudaSuccess ||
                fits <= 0) {
                cudaGetLastError();
                continue;
            }
            for (unsigned ch : chunks) {
                c->regs = regs;
                c->block = b;
                c->chunk = ch;
                float ms = 0.0f;
                if ((rc = timed(&ms))) goto done;
                if (best_ms < 0.0f || ms < best_ms) { best_ms = ms; best_block = b; best_chunk = ch; best_regs = regs; }
            }
        }
    }
    // finally the material source for the best shape: HU + table, or the
    // per-voxel (rho, SPR) grid (one more dependent load saved per step).
    // Both are timed twice and the faster minimum kept: the first run with
    // the grid also builds it, and the two are often within a few percent.
    if (best_ms > 0.0f) {
        c->regs = best_regs; c->block = best_block; c->chunk = best_chunk;
        float t_mat[2] = {-1.0f, -1.0f};
        for (int rep = 0; rep < 2; ++rep) {
            for (int m = 0; m < 2; ++m) {
                c->material_grid = m;
                float ms = 0.0f;
                if ((rc = timed(&ms))) goto done;
                if (t_mat[m] < 0.0f || ms < t_mat[m]) t_mat[m] = ms;
            }
        }
        best_mat = t_mat[1] < t_mat[0] ? 1 : 0;
        best_ms = t_mat[best_mat];
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->material_grid = rc ? keep_mat : best_mat;
    c->block = rc ? keep_block : best_block;
    c->chunk = rc ? keep_chunk : best_chunk;
    c->regs = rc ? keep_regs : best_regs;
    c->blocks_per_sm = keep_per_sm;
    if (!rc && best_ms < 0.0f) rc = fail(c, DOSE_ECUDA, "autotune: no launch shape could be timed");
    if (!rc && best) {
        best[0] = best_regs; best[1] = best_block; best[2] = best_chunk;
        best[3] = (int64_t)(best_ms * 1000.0f);
    }
    return rc;
}

}  // namespace

extern "C" {

int dose_autotune(dose_ctx *c, int phase, uint64_t n_histories, uint64_t sample_histories, uint64_t seed,
                  void *stream, int64_t best[4])
{
    if (!c) return fail(nullptr, DOSE_EINVAL, "ctx is NULL");
    if (sample_histories == 0 || sample_histories > n_histories)
        return fail(c, DOSE_EINVAL, "sample must be in 1..n_histories");
    cudaStream_t st = S(stream);
    dose_job j;
    j.ctx = c; j.phase = phase; j.n_histories = n_histories; j.seed = seed; j.spr_scale = 1.0f;
    j.shift_mm[0] = j.shift_mm[1] = j.shift_mm[2] = 0.0f;
    // allocate the phase's histories once; each trial then only transports
    j.flags = DOSE_JOB_CLEAR; j.hist_begin = 0; j.hist_end = 0;
    int rc = dose_run_batch(&j, 1, stream);
    if (!rc) {
        j.flags = 0; j.hist_begin = 0; j.hist_end = sample_histories;
        rc = tune_shapes(c, st, true, [&] { return dose_run_batch(&j, 1, stream); }, best);
    }
    if (phase >= 0 && phase < c->g->n_phases) c->ph[phase].has_dose = false;
    return rc;
}

int dose_autotune_batch(const dose_job *jobs, int n_jobs, uint64_t sample_histories, void *stream, int64_t best[4])
{
    if (!jobs || n_jobs <= 0 || !jobs[0].ctx) return fail(nullptr, DOSE_EINVAL, "no jobs");
    dose_ctx *c0 = jobs[0].ctx;
    if (sample_histories == 0) return fail(c0, DOSE_EINVAL, "sample_histories must be positive");
    unsigned long long total = 0;
    for (int k = 0; k < n_jobs; ++k) {
        if (!jobs[k].ctx) return fail(c0, DOSE_EINVAL, "job %d has no context", k);
        if (jobs[k].hist_end < jobs[k].hist_begin) return fail(c0, DOSE_EINVAL, "job %d: empty history range", k);
        total += jobs[k].hist_end - jobs[k].hist_begin;
    }
    if (total == 0) return fail(c0, DOSE_EINVAL, "the batch has no histories");
    // allocate each (context, phase) once, then time samples of every job:
    // job k transports the first ceil(sample x its share) histories of its range
    std::vector<dose_job> clear, sample;
    for (int k = 0; k < n_jobs; ++k) {
        bool seen = false;
        for (const auto &q : clear) seen |= q.ctx == jobs[k].ctx && q.phase == jobs[k].phase;
        if (!seen) {
            dose_job q = jobs[k];
            q.flags = DOSE_JOB_CLEAR; q.hist_begin = 0; q.hist_end = 0;
            clear.push_back(q);
        }
        const unsigned long long cnt = jobs[k].hist_end - jobs[k].hist_begin;
        if (!cnt) continue;
        dose_job q = jobs[k];
        q.flags = 0;
        const long double share = (long double)sample_histories * cnt / total;
        q.hist_end = q.hist_begin + std::min<unsigned long long>(cnt, (unsigned long long)std::ceil(share));
        sample.push_back(q);
    }
    int rc = dose_run_batch(clear.data(), (int)clear.size(), stream);
    if (rc) return rc;
    const bool single = sample.size() == 1;
    rc = tune_shapes(c0, S(stream), single,
                     [&] { return dose_run_batch(sample.data(), (int)sample.size(), stream); }, best);
    for (const auto &q : clear) {
        q.ctx->ph[q.phase].has_dose = false;
        if (rc) continue;
        q.ctx->regs = c0->regs; q.ctx->block = c0->block; q.ctx->chunk = c0->chunk;
        q.ctx->material_grid = c0->material_grid;
    }
    return rc;
}

int dose_run_4d(dose_ctx *c, uint64_t n_histories_per_phase, uint64_t seed, float spr_scale,
                const float shift_mm[3], int ref_phase, const int nsub[3], const float *dvf,
                int dvf_on_device, const uint8_t *mask, int mask_on_device, void *stream)
{
    if (!c) return fail(nullptr, DOSE_EINVAL, "ctx is NULL");
    if (!c->have_plan) return fail(c, DOSE_ESTATE, "no spots loaded");
    if (n_histories_per_phase == 0) return fail(c, DOSE_EINVAL, "n_histories_per_phase is 0");
    const int P = c->g->n_phases;
    if (ref_phase < 0 || ref_phase >= P) return fail(c, DOSE_EINVAL, "ref_phase out of range");
    int rc;
    if ((rc = use_device(c))) return rc;
    cudaStream_t st = S(stream);
    // per-phase proton totals of the subplans (skip phases with none)
    std::vector<unsigned long long> pp((size_t)P * c->n_spots);
    CK(c, cudaMemcpyAsync(pp.data(), c->pp, pp.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    if ((rc = sync_stream(c, st))) return rc;
    if ((rc = ensure_results(c, st))) return rc;
    std::vector<dose_job> jobs;
    for (int p = 0; p < P; ++p) {
        unsigned long long w = 0;
        for (int s = 0; s < c->n_spots; ++s) w += pp[(size_t)p * c->n_spots + s];
        if (w == 0) {
            CK(c, cudaMemsetAsync(c->ph[p].dose, 0, c->g->nvox * sizeof(float), st));
            c->ph[p].has_dose = true;
            continue;
        }
        dose_job j;
        j.ctx = c; j.phase = p; j.flags = DOSE_JOB_CLEAR | DOSE_JOB_FINISH;
        j.n_histories = n_histories_per_phase; j.hist_begin = 0; j.hist_end = n_histories_per_phase;
        j.seed = seed; j.spr_scale = spr_scale;
        for (int k = 0; k < 3; ++k) j.shift_mm[k] = shift_mm ? shift_mm[k] : 0.0f;
        jobs.push_back(j);
    }
    if (!jobs.empty() && (rc = dose_run_batch(jobs.data(), (int)jobs.size(), stream))) return rc;
    return dose_accumulate_subvoxel(c, ref_phase, nsub, dvf, dvf_on_device, mask, mask_on_device, 0, stream);
}

int dose_set_phase_dose(dose_ctx *c, int phase, const float *dose, int on_device, void *stream)
{
    if (!c) return fail(nullptr, DOSE_EINVAL, "ctx is NULL");
    if (!dose) return fail(c, DOSE_EINVAL, "dose is NULL");
    if (phase < 0 || phase >= c->g->n_phases) return fail(c, DOSE_EINVAL, "phase %d out of range", phase);
    int rc;
    if ((rc = use_device(c))) return rc;
    if ((rc = ensure_results(c, S(stream)))) return rc;
    PhaseState &P = c->ph[phase];
    CK(c, cudaMemcpyAsync(P.dose, dose, c->g->nvox * sizeof(float),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S(stream)));
    P.has_dose = true;
    c->have_accum = false;
    return DOSE_OK;
}

int dose_accumulate_subvoxel(dose_ctx *c, int ref_phase, const int nsub[3], const float *dvf,
                             int dvf_on_device, const uint8_t *mask, int mask_on_device, int method,
                             void *stream)
{
    if (!c) return fail(nullptr, DOSE_EINVAL, "ctx is NULL");
    if (method != 0 && method != 1) return fail(c, DOSE_EINVAL, "method must be 0 (EMTM) or 1 (DIM)");
    const Grid &g = *c->g;
    if (ref_phase < 0 || ref_phase >= g.n_phases) return fail(c, DOSE_EINVAL, "ref_phase out of range");
    if (!nsub || nsub[0] < 1 || nsub[1] < 1 || nsub[2] < 1 || nsub[0] > 64 || nsub[1] > 64 || nsub[2] > 64)
        return fail(c, DOSE_EINVAL, "nsub must be 3 values in 1..64");
    for (int p = 0; p < g.n_phases; ++p)
        if (!c->ph[p].has_dose) return fail(c, DOSE_ESTATE, "phase %d has no dose", p);
    int rc;
    if ((rc = use_device(c))) return rc;
    const size_t nvox = (size_t)g.nvox, P = (size_t)g.n_phases;
    if (!c->accum && (rc = dalloc_t(c, &c->accum, nvox))) return rc;
    if (method == 0 && !c->em) {
        if ((rc = dalloc_t(c, &c->em, 2 * P * nvox)) || (rc = dalloc_t(c, &c->maxbits, P)) ||
            (rc = dalloc_t(c, &c->emtm_stats, 4)))
            return rc;
    }
    cudaStream_t st = S(stream);
    const float *dvf_dev = dvf;
    const uint8_t *mask_dev = mask;
    if (dvf && !dvf_on_device) {
        if (!c->dvf_buf && (rc = dalloc_t(c, &c->dvf_buf, P * 3 * nvox))) return rc;
        CK(c, cudaMemcpyAsync(c->dvf_buf, dvf, P * 3 * nvox * sizeof(float), cudaMemcpyHostToDevice, st));
        dvf_dev = c->dvf_buf;
    }
    if (mask && !mask_on_device) {
        if (!c->mask_buf && (rc = dalloc_t(c, &c->mask_buf, nvox))) return rc;
        CK(c, cudaMemcpyAsync(c->mask_buf, mask, nvox, cudaMemcpyHostToDevice, st));
        mask_dev = c->mask_buf;
    }
    if (!c->reach && (rc = dalloc_t(c, &c->reach, P * kReachWords))) return rc;
    int sms = 0;
    CK(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g.device));
    CK(c, cudaMemsetAsync(c->reach, 0, P * kReachWords * sizeof(unsigned), st));
    ReachArgs ra;
    ra.dose = c->dose_all; ra.rho = method == 0 ? g.rho : nullptr; ra.dvf = dvf_dev;
    ra.reach = c->reach; ra.maxbits = nullptr;
    ra.nx = g.n[0]; ra.ny = g.n[1]; ra.nz = g.n[2]; ra.ref = ref_phase;
    if (method == 1) {
        k_reach<<<dim3((unsigned)(2 * sms), (unsigned)P), 256, 0, st>>>(ra);
        CK(c, cudaGetLastError());
        DimArgs a;
        a.dose = c->dose_all; a.dvf = dvf_dev; a.mask = mask_dev; a.accum = c->accum;
        a.nx = g.n[0]; a.ny = g.n[1]; a.nz = g.n[2];
        a.idx = 1.0f / g.d[0]; a.idy = 1.0f / g.d[1]; a.idz = 1.0f / g.d[2];
        a.nsx = nsub[0]; a.nsy = nsub[1]; a.nsz = nsub[2];
        a.ref = ref_phase; a.n_phases = (int)P;
        a.reach = c->reach;
        k_dim<<<(unsigned)((nvox + 255) / 256), 256, 0, st>>>(a);
        CK(c, cudaGetLastError());
        c->have_accum = true;
        c->accum_method = 1;
        return DOSE_OK;
    }
    CK(c, cudaMemsetAsync(c->maxbits, 0, P * sizeof(unsigned), st));
    CK(c, cudaMemsetAsync(c->emtm_stats, 0, 4 * sizeof(unsigned long long), st));
    EmtmArgs a;
    a.dose = c->dose_all; a.rho = g.rho; a.mask = mask_dev;
    a.E = c->em; a.M = c->em + P * nvox; a.maxbits = c->maxbits; a.reach = c->reach; a.stats = c->emtm_stats;
    a.accum = c->accum;
    a.nx = g.n[0]; a.ny = g.n[1]; a.nz = g.n[2];
    a.dx = g.d[0]; a.dy = g.d[1]; a.dz = g.d[2];
    a.nsx = nsub[0]; a.nsy = nsub[1]; a.nsz = nsub[2];
    a.ref = ref_phase; a.n_phases = (int)P;
    ra.maxbits = c->maxbits;
    k_reach<<<dim3((unsigned)(2 * sms), (unsigned)P), 256, 0, st>>>(ra);
    CK(c, cudaGetLastError());
    a.dvf4 = nullptr; a.phase = 0;
    a.idx = 1.0f / g.d[0]; a.idy = 1.0f / g.d[1]; a.idz = 1.0f / g.d[2];
    // grid-stride launches: the voxels within reach are not known on the host
    int per_sm = 0;
    CK(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_emtm, 256, 0));
    const unsigned grid = (unsigned)std::min<size_t>((nvox + 255) / 256, (size_t)sms * std::max(per_sm, 1));
    k_emtm_zero<<<dim3((unsigned)(4 * sms), (unsigned)P), 256, 0, st>>>(a);
    CK(c, cudaGetLastError());
    if (dvf_dev) {
        if (!c->dvf4 && (rc = dalloc_t(c, &c->dvf4, nvox))) return rc;
        for (int S = 0; S < (int)P; ++S) {
            if (S == ref_phase) continue;
            k_dvf4<<<grid, 256, 0, st>>>(dvf_dev + (size_t)S * 3 * nvox, c->dvf4, c->reach + (size_t)S * kReachWords,
                                         a.nx, a.ny, a.nz, a.idx, a.idy, a.idz);
            a.dvf4 = c->dvf4; a.phase = S;
            k_emtm<<<dim3(grid, 1), 256, 0, st>>>(a);
            CK(c, cudaGetLastError());
        }
    } else {
        k_emtm<<<dim3(grid, (unsigned)P), 256, 0, st>>>(a);
        CK(c, cudaGetLastError());
    }
    const size_t sum_smem = P * 8 * sizeof(int);
    if (sum_smem > 48 * 1024)
        CK(c, cudaFuncSetAttribute(k_emtm_sum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sum_smem));
    k_emtm_sum<<<1216, 256, sum_smem, st>>>(a);
    CK(c, cudaGetLastError());
    c->have_accum = true;
    c->accum_method = 0;
    return DOSE_OK;
}

int dose_decode_dvf(dose_ctx *c, const dose_dvf_grid *grid, const float *translation,
                    int translation_on_device, float *dvf_out, uint8_t *mask_inout, void *stream)
{
    if (!c) return fail(nullptr, DOSE_EINVAL, "ctx is NULL");
    if (!grid || !translation || !dvf_out) return fail(c, DOSE_EINVAL, "grid, translation and dvf_out are required");
    const dose_dvf_grid &G = *grid;
    for (int k = 0; k < 3; ++k) {
        if (G.n[k] < 1) return fail(c, DOSE_EINVAL, "grid size must be positive");
        if (!(G.spacing_mm[k] > 0.0f)) return fail(c, DOSE_EINVAL, "grid spacing must be positive");
    }
    double uu = 0, vv = 0, uv = 0;
    for (int k = 0; k < 3; ++k) {
        uu += (double)G.row_cos[k] * G.row_cos[k];
        vv += (double)G.col_cos[k] * G.col_cos[k];
        uv += (double)G.row_cos[k] * G.col_cos[k];
    }
    if (std::fabs(uu - 1.0) > 1e-4 || std::fabs(vv - 1.0) > 1e-4 || std::fabs(uv) > 1e-4)
        return fail(c, DOSE_EINVAL, "row and column direction cosines must be orthonormal");
    for (void *ptr : {(void *)dvf_out, (void *)mask_inout}) {
        if (!ptr) continue;
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(c, DOSE_EINVAL, "dvf_out and mask_inout must be device memory");
        }
    }
    int rc;
    if ((rc = use_device(c))) return rc;
    const Grid &g = *c->g;
    const size_t ng = (size_t)G.n[0] * G.n[1] * G.n[2];
    if (ng > (size_t)INT32_MAX) return fail(c, DOSE_EINVAL, "registration grid has 2^31 voxels or more");
    cudaStream_t st = S(stream);
    if (ng > c->dvfgrid_cap) {
        if (c->dvfgrid_e) { dfree(c, c->dvfgrid_e); c->dvfgrid_e = nullptr; }
        if (c->dvfgrid_delta) { dfree(c, c->dvfgrid_delta); c->dvfgrid_delta = nullptr; }
        c->dvfgrid_cap = 0;
        if ((rc = dalloc_t(c, &c->dvfgrid_e, 3 * ng)) || (rc = dalloc_t(c, &c->dvfgrid_delta, 3 * ng))) return rc;
        c->dvfgrid_cap = ng;
    }
    const float *delta = translation;
    if (!translation_on_device) {
        CK(c, cudaMemcpyAsync(c->dvfgrid_delta, translation, 3 * ng * sizeof(float), cudaMemcpyHostToDevice, st));
        delta = c->dvfgrid_delta;
    }
    DvfArgs a;
    for (int k = 0; k < 3; ++k) {
        a.gn[k] = G.n[k]; a.start[k] = G.start_mm[k]; a.sp[k] = G.spacing_mm[k];
        a.U[k] = G.row_cos[k]; a.V[k] = G.col_cos[k];
        a.n[k] = g.n[k]; a.d[k] = g.d[k]; a.origin[k] = g.origin[k];
    }
    const double U[3] = {G.row_cos[0], G.row_cos[1], G.row_cos[2]}, V[3] = {G.col_cos[0], G.col_cos[1], G.col_cos[2]};
    a.W[0] = (float)(U[1] * V[2] - U[2] * V[1]);
    a.W[1] = (float)(U[2] * V[0] - U[0] * V[2]);
    a.W[2] = (float)(U[0] * V[1] - U[1] * V[0]);
    for (int k = 0; k < 16; ++k) { a.pre[k] = G.pre[k]; a.post[k] = G.post[k]; }
    for (int r = 0; r < 3; ++r)
        for (int m = 0; m < 3; ++m) {
            double v = (r == m) ? -1.0 : 0.0;
            for (int t = 0; t < 3; ++t) v += (double)G.post[4 * r + t] * G.pre[4 * t + m];
            a.RR[3 * r + m] = (float)v;
        }
    a.delta = delta; a.e = c->dvfgrid_e; a.out = dvf_out; a.mask = mask_inout;
    k_dvf_grid<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(a);
    CK(c, cudaGetLastError());
    k_dvf_resample<<<(unsigned)((g.nvox + 255) / 256), 256, 0, st>>>(a);
    CK(c, cudaGetLastError());
    return DOSE_OK;
}

int dose_read(dose_ctx *c, int what, int phase, void *dst, size_t bytes, int dst_on_device, void *stream)
{
    if (!c) return fail(nullptr, DOSE_EINVAL, "ctx is NULL");
    if (!dst) return fail(c, DOSE_EINVAL, "dst is NULL");
    const Grid &g = *c->g;
    const size_t nvox = (size_t)g.nvox;
    const void *src = nullptr;
    size_t need = 0;
    auto phase_ok = [&] { return phase >= 0 && phase < g.n_phases; };
    switch (what) {
    case DOSE_PHASE_DOSE:
        if (!phase_ok()) return fail(c, DOSE_EINVAL, "phase out of range");
        if (!c->ph[phase].has_dose) return fail(c, DOSE_ESTATE, "phase %d has no dose", phase);
        src = c->ph[phase].dose; need = nvox * sizeof(float); break;
    case DOSE_DENSITY:
        if (!phase_ok()) return fail(c, DOSE_EINVAL, "phase out of range");
        src = g.rho + (size_t)phase * nvox; need = nvox * sizeof(float); break;
    case DOSE_ACCUM:
        if (!c->have_accum) return fail(c, DOSE_ESTATE, "no accumulated dose");
        src = c->accum; need = nvox * sizeof(float); break;
    case DOSE_TALLY_I64:
        if (!phase_ok()) return fail(c, DOSE_EINVAL, "phase out of range");
        if (!c->ph[phase].tally || !c->ph[phase].allocated) return fail(c, DOSE_ESTATE, "phase %d was not run", phase);
        src = c->ph[phase].tally; need = nvox * sizeof(unsigned long long); break;
    case DOSE_SUBPLAN:
        if (!c->have_plan) return fail(c, DOSE_ESTATE, "no plan");
        src = c->pp; need = (size_t)g.n_phases * c->n_spots * sizeof(unsigned long long); break;
    case DOSE_ENERGY_LEDGER:
    case DOSE_STATUS:
        if (!phase_ok()) return fail(c, DOSE_EINVAL, "phase out of range");
        if (!c->ph[phase].ledger || !c->ph[phase].allocated) return fail(c, DOSE_ESTATE, "phase %d was not run", phase);
        src = c->ph[phase].ledger;
        need = what == DOSE_STATUS ? sizeof(int32_t) : LED_WORDS * sizeof(unsigned long long);
        break;
    case DOSE_START_PHASE:
        if (!c->have_plan) return fail(c, DOSE_ESTATE, "no plan");
        src = c->start_phase; need = c->n_fields * sizeof(int32_t); break;
    case DOSE_FIELD_END_NS:
        if (!c->have_plan) return fail(c, DOSE_ESTATE, "no plan");
        src = c->field_end; need = c->n_fields * sizeof(int64_t); break;
    case DOSE_EMTM_STATS:
        if (!c->have_accum || c->accum_method != 0) return fail(c, DOSE_ESTATE, "no energy/mass-transfer accumulation");
        src = c->emtm_stats; need = 4 * sizeof(unsigned long long); break;
    case DOSE_DELIVERY:
        if (!c->have_plan || !c->have_delivery) return fail(c, DOSE_ESTATE, "no delivery simulation ran");
        src = c->tl_used; need = sizeof(dose_delivery); break;
    case DOSE_HIST_PREFIX:
        if (!phase_ok()) return fail(c, DOSE_EINVAL, "phase out of range");
        if (!c->ph[phase].allocated || !c->ph[phase].prefix) return fail(c, DOSE_ESTATE, "phase %d was not run", phase);
        src = c->ph[phase].prefix; need = ((size_t)c->n_spots + 1) * sizeof(unsigned long long); break;
    default:
        return fail(c, DOSE_EINVAL, "unknown selector %d", what);
    }
    if (bytes != need) return fail(c, DOSE_EINVAL, "selector %d needs %zu bytes, got %zu", what, need, bytes);
    int rc;
    if ((rc = use_device(c))) return rc;
    cudaStream_t st = S(stream);
    if (what == DOSE_STATUS) {
        if (dst_on_device) return fail(c, DOSE_EINVAL, "DOSE_STATUS is read into host memory only");
        unsigned long long led[LED_WORDS];
        CK(c, cudaMemcpyAsync(led, src, sizeof led, cudaMemcpyDeviceToHost, st));
        if ((rc = sync_stream(c, st))) return rc;
        *(int32_t *)dst = (led[LED_FLAGS] & FLAG_STEPLIMIT) ? DOSE_ESTEPLIMIT : DOSE_OK;
        return DOSE_OK;
    }
    CK(c, cudaMemcpyAsync(dst, src, need, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (!dst_on_device) return sync_stream(c, st);
    return DOSE_OK;
}

int dose_debug_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n, float *uniforms)
{
    if (!ctr || !key || !out || n <= 0 || n > (1 << 24)) return fail(nullptr, DOSE_EINVAL, "bad arguments");
    uint4 *dc = nullptr, *dout = nullptr;
    uint2 *dk = nullptr;
    float *du = nullptr;
    cudaError_t e = cudaMalloc(&dc, n * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMalloc(&dk, n * sizeof(uint2));
    if (e == cudaSuccess) e = cudaMalloc(&dout, n * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMalloc(&du, n * 6 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, n * sizeof(uint4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, n * sizeof(uint2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_debug_philox<<<(n + 255) / 256, 256>>>(dc, dk, dout, du, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, n * sizeof(uint4), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && uniforms) e = cudaMemcpy(uniforms, du, n * 6 * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(dc); cudaFree(dk); cudaFree(dout); cudaFree(du);
    if (e != cudaSuccess) return fail(nullptr, DOSE_ECUDA, "philox self-test: %s", cudaGetErrorString(e));
    return DOSE_OK;
}

int dose_debug_tables(const float *E, int n, float *out, void *stream)
{
    if (!E || !out || n <= 0 || n > (1 << 24)) return fail(nullptr, DOSE_EINVAL, "bad arguments");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, DOSE_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    DeviceTables tab;
    dose_ctx tmp;
    int rc = device_tables(&tmp, dev, &tab);
    if (rc) return fail(nullptr, rc, "%s", tmp.err.c_str());
    float *de = nullptr, *dout = nullptr;
    e = cudaMalloc(&de, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dout, n * 5 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(de, E, n * sizeof(float), cudaMemcpyHostToDevice, S(stream));
    if (e == cudaSuccess) {
        k_debug_tables<<<(n + 255) / 256, 256, 0, S(stream)>>>(tab.dev, tab.inv_ds, de, n, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, n * 5 * sizeof(float), cudaMemcpyDeviceToHost, S(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(S(stream));
    cudaFree(de); cudaFree(dout);
    if (e != cudaSuccess) return fail(nullptr, DOSE_ECUDA, "table self-test: %s", cudaGetErrorString(e));
    return DOSE_OK;
}

int dose_debug_spread(uint64_t n, uint32_t log2_strides, uint64_t *out)
{
    if (!out || n > (1ull << 26) || log2_strides > 16) return fail(nullptr, DOSE_EINVAL, "bad arguments");
    for (uint64_t w = 0; w < n; ++w) out[w] = spread_history(w, n, log2_strides);
    return DOSE_OK;
}

void dose_destroy(dose_ctx *c)
{
    if (!c) return;
    if (c->g) cudaSetDevice(c->g->device);
    cudaDeviceSynchronize();                 // nothing in flight uses the blocks below
    for (auto &o : c->owned) block_release(o.first, o.second);
    c->owned.clear();
    if (c->g && c->g->refs.fetch_sub(1) == 1) {
        const size_t n_all = (size_t)c->g->nvox * c->g->n_phases;
        block_release(c->g->hu, n_all * sizeof(int16_t));
        block_release(c->g->rho, n_all * sizeof(float));
        block_release(c->g->mat, n_all * sizeof(float2));
        delete c->g;
    }
    delete c;
}

}  // extern "C"
