// Kernel declarations shared between the engine's translation units.
#pragma once
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>
#include "dose.h"
#include "engine.cuh"

namespace dose {

// Record the message dose_last_error(NULL) returns on this thread.
void set_thread_error(const char *msg);
}  // namespace dose
struct dose_ctx;
namespace dose {
// nx, ny, nz, n_phases of a context's grid.
void grid_info(const dose_ctx *c, int dims[4]);
// Give a phase zero dose (a phase its plan does not reach).
int set_phase_zero(dose_ctx *c, int phase, void *stream);
// Give dst (a view of src's grid) src's plan and delivery result: the plan
// arrays, the subplan, start phases, field ends and field beams are copied
// on the stream, so the timeline does not run again.
int copy_plan(dose_ctx *dst, const dose_ctx *src, void *stream);

__global__ void k_density(const int16_t *hu, float *rho, long long n, const Tables *tab);
__global__ void k_material(const int16_t *hu, float2 *m, long long n, const Tables *tab);
__global__ void k_alloc(const AllocJob *jobs);
// The transport kernels (csrc/transport.cu), reached through
// transport_kernel() and transport_launch().  mode: one job as a kernel
// parameter (kLaunchSingle; the launch gives transport_smem(1) +
// birth_smem(block) bytes of shared memory), a table of jobs whose
// per-step fields (see jobs_share_step_fields) come from the parameter
// `job0` (kLaunchShared), a table of jobs that share only the grid,
// physics and step limit (see jobs_share_geometry), which come from `job0`
// while round keys and SPR scale come from each job (kLaunchGeom), or a
// general table (kLaunchTable).  For the table modes, stage != 0: the
// launch gives transport_smem(n_jobs) +
// birth_smem(block) bytes and the job table is staged in shared memory;
// 0: transport_smem(kMaxStagedJobs + 1) + birth_smem(block) (tables only)
// and the jobs are read from global memory.  regs: 1 = the 64-register
// build (blocks up to 1024 threads), 0 = up to 128 registers (blocks up to
// 512).  spec: kSpecGeneric reads each job's physics mask and material
// source; kSpecFullGrid and kSpecFullHu are built for jobs that all have
// every physics process on and, respectively, all have a per-voxel (rho,
// SPR) grid or all read HU + table (transport_spec() says which applies).
enum { kLaunchTable = 0, kLaunchSingle = 1, kLaunchShared = 2, kLaunchGeom = 3 };
enum { kSpecGeneric = 0, kSpecFullGrid = 1, kSpecFullHu = 2 };
struct TransportLaunch {
    int mode, regs, spec;
    unsigned grid, block;
    size_t smem;
    cudaStream_t stream;
    const TJob *job0;                   // host: the job (single) or the shared fields (shared, geom)
    const TJob *d_jobs;                 // device table (the table modes)
    int n_jobs;
    unsigned long long total;           // work items
    unsigned long long *counter;        // device work counter, zero at launch
    const Tables *tab;
    float inv_ds;
    unsigned chunk;
    int stage;
};
// The jobs of a batch with at least this many work items run in single-job
// launches of their own, after one launch shared by the others: the
// single-job step is a few per cent cheaper, and a launch's tail (its
// longest histories finishing on a part-idle GPU) costs about 0.7 ms, so
// a launch of its own pays only for jobs of tens of milliseconds and more.
constexpr unsigned long long kSplitWork = 1ull << 25;
// The most specialised kernel every job of the launch satisfies.
int transport_spec(const TJob *jobs, int n);
const void *transport_kernel(int mode, int regs, int spec);
cudaError_t transport_launch(const TransportLaunch &L);
// True when every job agrees with the first on the per-step fields other
// than the SPR scale and the round keys: grid and voxel sizes, physics,
// step limit (kLaunchGeom).
inline bool jobs_share_geometry(const TJob *jobs, int n)
{
    constexpr size_t a = offsetof(TJob, spr_scale), b = offsetof(TJob, idx), e = offsetof(TJob, rk);
    for (int j = 1; j < n; ++j)
        if (std::memcmp(&jobs[j], &jobs[0], a) != 0 ||
            std::memcmp(reinterpret_cast<const char *>(&jobs[j]) + b, reinterpret_cast<const char *>(&jobs[0]) + b,
                        e - b) != 0)
            return false;
    return true;
}
// True when every job agrees with the first on the per-step fields (the
// first kStepFieldBytes bytes of a TJob).
inline bool jobs_share_step_fields(const TJob *jobs, int n)
{
    for (int j = 1; j < n; ++j)
        if (std::memcmp(&jobs[j], &jobs[0], kStepFieldBytes) != 0) return false;
    return true;
}
// Every transport kernel accepts up to kSmemTransportMax + birth_smem(1024)
// bytes of dynamic shared memory (set once per device before a launch).
cudaError_t transport_allow_smem();
__global__ void k_normalise(const NormJob *jobs);
__global__ void k_debug_philox(const uint4 *ctr, const uint2 *key, uint4 *out, float *uni, int n);
__global__ void k_debug_tables(const Tables *tab, float inv_ds, const float *e, int n, float *out);

// Delivery parameters that keep the clock moving: every fill and every gate
// window delivers at least one proton (shortest cycle mu - 6 sigma, the
// Irwin-Hall bound, at least N ns).  Shared by the host checks and the
// kernel's check of sampled trial deliveries.
__host__ __device__ inline bool delivery_ok(const dose_delivery &d)
{
    if (d.n_phases <= 0 || d.repaints <= 0 || d.period_ns <= 0 || d.rate_protons_per_s == 0 ||
        d.period_sigma_ns < 0 || d.period_sigma_ns > (1ll << 38) || d.spot_switch_ns < 0 ||
        d.layer_switch_ns < 0 || d.discard_ns < 0 || d.start_phase >= d.n_phases || d.extraction_limit_ns < 0)
        return false;
    if (d.max_protons_per_paint > 0 && d.repaints != 1) return false;
    if (d.synchrotron != 0 && d.synchrotron != 1) return false;
    const long long tmin = d.period_ns - 6 * d.period_sigma_ns;
    if (tmin < d.n_phases) return false;
    const long long tph_min = tmin / d.n_phases;
    const long long proton_ns = (long long)((1000000000ull + d.rate_protons_per_s - 1) / d.rate_protons_per_s);
    if (d.gated) {
        if (d.gate_first < 0 || d.gate_last >= d.n_phases || d.gate_first > d.gate_last) return false;
        const long long window = (long long)(d.gate_last - d.gate_first + 1) * tph_min;
        if (d.discard_ns >= window) return false;
        if (d.synchrotron && window - d.discard_ns < proton_ns) return false;
    }
    if (d.synchrotron && d.extraction_limit_ns > 0 && d.extraction_limit_ns < proton_ns) return false;
    return true;
}

struct TimelineArgs {                // one trial (or the single delivery) of a plan
    const unsigned long long *protons;
    const int *layer;
    const int *field;
    int n_spots, n_fields;
    dose_delivery d;                 // the delivery, or the mean of the trials
    const dose_delivery_spread *spread;   // device; null: d as given
    unsigned long long trial;
    unsigned long long *pp;          // n_phases x n_spots, zeroed by the caller
    long long *field_end;            // n_fields
    int *start_out;                  // n_fields
    dose_delivery *used;             // the delivery the clock ran (sampled for trials)
    int *status;                     // 0; 1 sampled delivery invalid; 2 no progress; 3 clock overflow
};
// One block per trial, a thread per field; dynamic shared memory
// 13 B per spot (the plan's protons, layers and fields).
__global__ void k_timeline(const TimelineArgs *args);

// What an accumulation can reach, per source phase: a record of
// kReachWords words, zeroed before k_reach fills it.  Words 0-2 hold the
// bitwise NOT of the lowest x, y, z index of a voxel that carries dose
// (rho > 0 and D > 0 for the EMTM, D != 0 for the DIM), words 3-5 one past
// the highest (0: no such voxel), words 6-8 the bits of max |u| per axis
// (mm) of the phase's field (0 without a field).  reach_box grows it into
// the voxels the accumulation has to visit.
constexpr int kReachWords = 12;
struct ReachArgs {
    const float *dose;               // n_phases x nvox
    const float *rho;                // n_phases x nvox (EMTM), or null: the DIM's D != 0
    const float *dvf;                // n_phases x 3 x nvox (mm), or null
    unsigned *reach;                 // n_phases x kReachWords, zeroed
    unsigned *maxbits;               // n_phases: bits of max(rho D) (EMTM), or null
    int nx, ny, nz;
    int ref;
};
__global__ void k_reach(ReachArgs a);

struct EmtmArgs {
    const float *dose;               // n_phases x nvox
    const float *rho;                // n_phases x nvox
    const uint8_t *mask;             // nvox or null
    unsigned long long *E, *M;       // n_phases x nvox each (slot of the reference unused)
    unsigned *maxbits;               // n_phases: bits of max(rho D) per phase
    const unsigned *reach;           // n_phases x kReachWords (k_reach)
    unsigned long long *stats;       // 4: pushed, dropped, atomic pairs, reserved
    float *accum;                    // nvox
    int nx, ny, nz;
    float dx, dy, dz;
    int nsx, nsy, nsz;
    int ref, n_phases;
    const float4 *dvf4;              // one source phase's field, interleaved, or null (identity)
    int phase;                       // that source phase (grid.y is the phase when dvf4 is null)
    float idx, idy, idz;             // 1 / voxel size, rounded to FP32
};
// The field nodes the source voxels of reach_box(reach, 2) read (that box
// grown by one voxel), interleaved; every other node of dst is left as is.
__global__ void k_dvf4(const float *src, float4 *dst, const unsigned *reach, int nx, int ny, int nz,
                       float idx, float idy, float idz);
__global__ void k_emtm(EmtmArgs a);
__global__ void k_emtm_zero(EmtmArgs a);
__global__ void k_emtm_sum(EmtmArgs a);        // dynamic shared memory: 32 B per phase

struct DimArgs {
    const float *dose;               // n_phases x nvox
    const float *dvf;                // n_phases x 3 x nvox (reference -> phase, mm), or null
    const uint8_t *mask;             // nvox or null
    float *accum;                    // nvox
    int nx, ny, nz;
    float idx, idy, idz;             // 1 / voxel sizes (mm -> voxels)
    int nsx, nsy, nsz;
    int ref, n_phases;
    const unsigned *reach;           // n_phases x kReachWords (k_reach over D != 0)
};
__global__ void k_dim(DimArgs a);

struct DvfArgs {
    int gn[3];                       // registration grid voxels
    float start[3], sp[3];           // centre of grid voxel 0, spacing (mm)
    float U[3], V[3], W[3];          // row, column, depth direction cosines (W = U x V)
    float pre[16], post[16];         // rigid transforms, row-major
    float RR[9];                     // R_post R_pre - I
    const float *delta;              // grid voxels x 3 (interleaved), mm
    float *e;                        // 3 x grid voxels: r_f - r0
    int n[3];                        // CT grid
    float d[3], origin[3];
    float *out;                      // 3 x nvox displacement, mm
    uint8_t *mask;                   // nvox, cleared outside the grid hull, or null
};
__global__ void k_dvf_grid(DvfArgs a);
__global__ void k_dvf_resample(DvfArgs a);

}  // namespace dose
