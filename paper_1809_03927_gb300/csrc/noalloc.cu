// dose_run_phase_noalloc: the Monte Carlo dose of one static plan (every
// spot on one CT grid) without allocating device memory.
//
// Some callers cannot call cudaMalloc: code running under a memory manager
// that owns the whole device (a framework's caching allocator, a plug-in
// given a fixed budget, a real-time service that forbids allocation after
// start-up).  They pass their own input and output buffers; everything else
// the kernels need -- the 64-bit tally, the spot table, the allocation
// arrays, the ledger, the work counter, the allocation descriptor and the
// lookup tables -- lives in one file-scope static __device__ array of fixed
// size, which every GPU that loads the library keeps until the process
// exits.  The transport job itself travels in the launch's parameters.
#include <cuda_runtime.h>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "dose.h"
#include "engine.cuh"
#include "kernels.h"

using namespace dose;

namespace {

// ---- the scratch array and its layout -------------------------------------
constexpr size_t kMaxVoxels = DOSE_NOALLOC_MAX_VOXELS;
constexpr size_t kMaxSpots = DOSE_NOALLOC_MAX_SPOTS;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffTally = 0;
constexpr size_t kOffSpot = align256(kOffTally + kMaxVoxels * sizeof(unsigned long long));
constexpr size_t kOffProtons = align256(kOffSpot + kMaxSpots * sizeof(float4));
constexpr size_t kOffPrefix = align256(kOffProtons + kMaxSpots * sizeof(unsigned long long));
constexpr size_t kOffRem = align256(kOffPrefix + (kMaxSpots + 1) * sizeof(unsigned long long));
constexpr size_t kOffWh = align256(kOffRem + kMaxSpots * sizeof(unsigned long long));
constexpr size_t kOffLedger = align256(kOffWh + kMaxSpots * sizeof(float));
constexpr size_t kOffCounter = align256(kOffLedger + LED_WORDS * sizeof(unsigned long long));
constexpr size_t kOffAlloc = align256(kOffCounter + 2 * sizeof(unsigned long long));
constexpr size_t kOffTables = align256(kOffAlloc + sizeof(AllocJob));
constexpr size_t kScratchBytes = align256(kOffTables + sizeof(Tables));

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// ---- per-device set-up: the array's device address and the tables --------
constexpr int kMaxDev = 64;
std::mutex g_mutex;
unsigned char *g_base[kMaxDev] = {};
Tables g_host_tab;
float g_inv_ds = 0.0f;
bool g_host_ready = false;
// Failures are reported through dose_last_error(NULL), like every call that
// has no context.
int fail(int code, const char *msg, cudaError_t e = cudaSuccess)
{
    char buf[256];
    if (e != cudaSuccess) snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
    else snprintf(buf, sizeof buf, "%s", msg);
    set_thread_error(buf);
    return code;
}

// Done on the first call on each device, with that device current: look up
// where the static array lives on this device (in host code its name is
// only a host-side stand-in) and fill its lookup tables.
int setup(int dev, unsigned char **base)
{
    std::lock_guard<std::mutex> lock(g_mutex);
    if (dev < 0 || dev >= kMaxDev) return fail(DOSE_ECUDA, "device index out of range");
    if (g_base[dev]) { *base = g_base[dev]; return DOSE_OK; }
    if (!g_host_ready) {
        build_tables(&g_host_tab, &g_inv_ds);
        g_host_ready = true;
    }
    unsigned char *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_scratch);
    if (e != cudaSuccess) return fail(DOSE_ECUDA, "cudaGetSymbolAddress", e);
    e = cudaMemcpy(p + kOffTables, &g_host_tab, sizeof(Tables), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(DOSE_ECUDA, "table upload", e);
    e = transport_allow_smem();
    if (e != cudaSuccess) return fail(DOSE_ECUDA, "cudaFuncSetAttribute", e);
    g_base[dev] = p;
    *base = p;
    return DOSE_OK;
}

// Dose from the tally with the density of each voxel taken from its HU
// through the calibration table (no density grid is kept): the same FP32
// density, the same FP64 factor and the same quotient (div64) as
// k_normalise, so the dose is bit for bit that of dose_run_phase.
__global__ void k_normalise_hu(const unsigned long long *__restrict__ tally,
                               unsigned long long *__restrict__ ledger, const int16_t *__restrict__ hu,
                               const Tables *__restrict__ tab, float *__restrict__ dose, long long nvox,
                               unsigned long long n_hist, double voxel_cm3)
{
    const unsigned long long W = ledger[LED_W];
    const double factor = (W == 0 || n_hist == 0) ? 0.0
        : (double)W / (double)n_hist * 1.602176634e-10 / (16777216.0 * voxel_cm3);
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned long long dep = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
        const unsigned long long t = tally[i];
        dep += t;
        const int h = min(max((int)hu[i], kHuMin), kHuMax);
        dose[i] = t ? (float)div64((double)t * factor, (double)tab->mat[h - kHuMin].x) : 0.0f;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) dep += __shfl_xor_sync(0xffffffffu, dep, o);
    if ((threadIdx.x & 31) == 0 && dep) atomicAdd(ledger + LED_DEP, dep);
}

}  // namespace

extern "C" {

int dose_run_phase_noalloc(const int16_t *hu, int nx, int ny, int nz, float dx_mm, float dy_mm,
                           float dz_mm, const float origin_mm[3], const float beam_dir[3],
                           const dose_spot *spots, int n_spots, uint64_t n_histories, uint64_t seed,
                           float *dose, uint64_t ledger_out[8], void *stream)
{
    if (!hu || !dose || !spots || !origin_mm || !beam_dir) return fail(DOSE_EINVAL, "NULL argument");
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(DOSE_EINVAL, "grid dimensions must be positive");
    const long long nvox = (long long)nx * ny * nz;
    if ((size_t)nvox > kMaxVoxels) return fail(DOSE_EINVAL, "grid of nx*ny*nz voxels exceeds DOSE_NOALLOC_MAX_VOXELS");
    if (!std::isfinite(origin_mm[0]) || !std::isfinite(origin_mm[1]) || !std::isfinite(origin_mm[2]))
        return fail(DOSE_EINVAL, "origin must be 3 finite values");
    if (n_spots <= 0 || (size_t)n_spots > kMaxSpots) return fail(DOSE_EINVAL, "spots must be in 1..DOSE_NOALLOC_MAX_SPOTS");
    if (n_histories == 0) return fail(DOSE_EINVAL, "n_histories is 0");
    if (!(dx_mm > 0 && dy_mm > 0 && dz_mm > 0) || !std::isfinite(dx_mm) || !std::isfinite(dy_mm) || !std::isfinite(dz_mm))
        return fail(DOSE_EINVAL, "voxel sizes must be positive and finite");
    int axis = -1, sign = 0, count = 0;
    for (int k = 0; k < 3; ++k) {
        if (beam_dir[k] == 1.0f || beam_dir[k] == -1.0f) { axis = k; sign = beam_dir[k] > 0 ? 1 : -1; ++count; }
        else if (beam_dir[k] != 0.0f) return fail(DOSE_EINVAL, "beam_dir must be a unit axis vector");
    }
    if (count != 1) return fail(DOSE_EINVAL, "beam_dir must be a unit axis vector");
    unsigned long long total = 0;
    for (int s = 0; s < n_spots; ++s) {
        if (total + spots[s].protons < total) return fail(DOSE_EINVAL, "total protons overflow 64 bits");
        total += spots[s].protons;
        if (!(spots[s].energy_MeV >= 1.0f && spots[s].energy_MeV <= 250.0f))
            return fail(DOSE_EINVAL, "spot energy outside 1..250 MeV");
        if (!(spots[s].sigma_mm >= 0.0f) || !std::isfinite(spots[s].sigma_mm) || !std::isfinite(spots[s].x_mm) ||
            !std::isfinite(spots[s].y_mm))
            return fail(DOSE_EINVAL, "spot position and sigma must be finite, sigma >= 0");
        if (spots[s].field != 0)
            return fail(DOSE_EINVAL, "every spot must belong to field 0 (one static field along beam_dir)");
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(DOSE_ECUDA, "cudaGetDevice", e);
    unsigned char *base = nullptr;
    int rc = setup(dev, &base);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    unsigned long long *tally = reinterpret_cast<unsigned long long *>(base + kOffTally);
    float4 *d_spot = reinterpret_cast<float4 *>(base + kOffSpot);
    unsigned long long *d_protons = reinterpret_cast<unsigned long long *>(base + kOffProtons);
    unsigned long long *d_ledger = reinterpret_cast<unsigned long long *>(base + kOffLedger);
    unsigned long long *d_counter = reinterpret_cast<unsigned long long *>(base + kOffCounter);
    const Tables *d_tab = reinterpret_cast<const Tables *>(base + kOffTables);

    // the spot table: staged through a fixed-size host buffer in chunks
    // (no allocation on either side)
    {
        float4 hs[256];
        unsigned long long hp[256];
        for (int s0 = 0; s0 < n_spots; s0 += 256) {
            const int m = n_spots - s0 < 256 ? n_spots - s0 : 256;
            for (int k = 0; k < m; ++k) {
                const dose_spot &q = spots[s0 + k];
                hs[k] = make_float4(q.x_mm, q.y_mm, q.energy_MeV, q.sigma_mm);
                hp[k] = q.protons;
            }
            e = cudaMemcpyAsync(d_spot + s0, hs, m * sizeof(float4), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_protons + s0, hp, m * sizeof(unsigned long long), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // hs/hp are reused
            if (e != cudaSuccess) return fail(DOSE_ECUDA, "spot upload", e);
        }
    }
    // everything that must start at zero: the tally of this grid, the
    // ledger and the work counter (the array keeps the last call's contents)
    e = cudaMemsetAsync(tally, 0, (size_t)nvox * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ledger, 0, LED_WORDS * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return fail(DOSE_ECUDA, "clear", e);

    AllocJob a;
    a.protons = d_protons;
    a.spot = d_spot;
    a.rem = reinterpret_cast<unsigned long long *>(base + kOffRem);
    a.prefix = reinterpret_cast<unsigned long long *>(base + kOffPrefix);
    a.wh = reinterpret_cast<float *>(base + kOffWh);
    a.ledger = d_ledger;
    a.n_spots = n_spots;
    a.n_hist = n_histories;
    // the transport job, as dose_run_phase describes it (default options)
    TJob t;
    t.hu = hu; t.matg = nullptr; t.tally = tally; t.ledger = d_ledger;
    t.spot = d_spot; t.wh = a.wh; t.prefix = a.prefix; t.n_spots = n_spots;
    t.nx = nx; t.ny = ny; t.nz = nz; t.dx = dx_mm; t.dy = dy_mm; t.dz = dz_mm;
    t.idx = 1.0f / dx_mm; t.idy = 1.0f / dy_mm; t.idz = 1.0f / dz_mm;
    t.o[0] = origin_mm[0]; t.o[1] = origin_mm[1]; t.o[2] = origin_mm[2];
    t.spot_dir = nullptr;
    t.beam_axis = axis; t.beam_sign = sign;
    t.spr_scale = 1.0f; t.physics = DOSE_PHYS_ALL; t.max_steps = 20000;
    t.key0 = (unsigned)seed; t.key1 = (unsigned)(seed >> 32);
    for (int r = 0; r < 10; r += 2)   // Philox round keys: key + r x the Weyl increments
        t.rk[r >> 1] = make_uint4(t.key0 + (unsigned)r * 0x9E3779B9u, t.key1 + (unsigned)r * 0xBB67AE85u,
                                  t.key0 + (unsigned)(r + 1) * 0x9E3779B9u, t.key1 + (unsigned)(r + 1) * 0xBB67AE85u);
    t.stream = 0;
    t.hist_begin = 0; t.work_begin = 0; t.n_work = n_histories; t.spread_log2 = spread_for(nvox, n_histories);
    AllocJob *d_a = reinterpret_cast<AllocJob *>(base + kOffAlloc);
    e = cudaMemcpyAsync(d_a, &a, sizeof a, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);                   // a lives on this stack
    if (e != cudaSuccess) return fail(DOSE_ECUDA, "descriptor upload", e);

    k_alloc<<<1, 1024, 0, st>>>(d_a);
    int sms = 0, per_sm = 0;
    const size_t smem = transport_smem(1) + birth_smem(1024);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int spec = transport_spec(&t, 1);      // all physics, HU + table
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, transport_kernel(kLaunchSingle, 1, spec), 1024, smem);
    if (e != cudaSuccess || per_sm <= 0) return fail(DOSE_ECUDA, "transport launch set-up", e);
    TransportLaunch L;                            // the default launch shape: 64 registers, 1024 threads, chunk 32
    L.mode = kLaunchSingle; L.regs = 1; L.spec = spec;
    L.grid = (unsigned)(sms * per_sm); L.block = 1024; L.smem = smem; L.stream = st;
    L.job0 = &t; L.d_jobs = nullptr; L.n_jobs = 1;
    L.total = n_histories; L.counter = d_counter; L.tab = d_tab; L.inv_ds = g_inv_ds;
    L.chunk = 32; L.stage = 0;
    e = transport_launch(L);
    if (e != cudaSuccess) return fail(DOSE_ECUDA, "launch", e);
    k_normalise_hu<<<304, 256, 0, st>>>(tally, d_ledger, hu, d_tab, dose, nvox, n_histories,
                                        (double)dx_mm * dy_mm * dz_mm / 1000.0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DOSE_ECUDA, "launch", e);
    // wait for the work, then report the ledger and the step-limit flag
    unsigned long long led[LED_WORDS];
    e = cudaMemcpyAsync(led, d_ledger, sizeof led, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(DOSE_ECUDA, "ledger read", e);
    if (ledger_out) std::memcpy(ledger_out, led, sizeof led);
    if (led[LED_FLAGS] & FLAG_STEPLIMIT)
        return fail(DOSE_ESTEPLIMIT, "a history reached the step limit (its energy is counted as escaped)");
    return DOSE_OK;
}

}  // extern "C"
