// Kernel declarations shared between the engine's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
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

__global__ void k_density(const int16_t *hu, float *rho, long long n, const Tables *tab);
__global__ void k_alloc(const AllocJob *jobs);
__global__ void k_transport(const TJob *jobs, int n_jobs, unsigned long long total,
                            unsigned long long *counter, const Tables *gtab, float inv_ds,
                            unsigned chunk);
__global__ void k_transport_r64(const TJob *jobs, int n_jobs, unsigned long long total,
                                unsigned long long *counter, const Tables *gtab, float inv_ds,
                                unsigned chunk);
__global__ void k_normalise(const NormJob *jobs);
__global__ void k_debug_philox(const uint4 *ctr, const uint2 *key, uint4 *out, float *uni, int n);
__global__ void k_debug_tables(const Tables *tab, float inv_ds, const float *e, int n, float *out);

struct TimelineArgs {
    const unsigned long long *protons;
    const int *layer;
    const int *field;
    int n_spots;
    int n_phases, start_phase, gated, gate_first, gate_last, repaints;
    long long tph, spot_switch, layer_switch, discard;
    unsigned long long rate, seed;
    unsigned long long *pp;          // n_phases x n_spots, zeroed by the caller
    long long *field_end;            // n_fields
    int *start_out;                  // n_fields
    int n_fields;
};
__global__ void k_timeline(TimelineArgs a);

struct EmtmArgs {
    const float *dose;               // n_phases x nvox
    const float *rho;                // n_phases x nvox
    const float *dvf;                // n_phases x 3 x nvox, or null
    const uint8_t *mask;             // nvox or null
    unsigned long long *E, *M;       // n_phases x nvox each (slot of the reference unused)
    unsigned *maxbits;               // n_phases: bits of max(rho D) per phase
    unsigned long long *stats;       // 4: pushed, dropped, atomic pairs, reserved
    float *accum;                    // nvox
    int nx, ny, nz;
    float dx, dy, dz;
    int nsx, nsy, nsz;
    int ref, n_phases;
};
__global__ void k_emtm_max(EmtmArgs a);
__global__ void k_emtm(EmtmArgs a);
__global__ void k_emtm_sum(EmtmArgs a);

struct DimArgs {
    const float *dose;               // n_phases x nvox
    const float *dvf;                // n_phases x 3 x nvox (reference -> phase, mm), or null
    const uint8_t *mask;             // nvox or null
    float *accum;                    // nvox
    int nx, ny, nz;
    float idx, idy, idz;             // 1 / voxel sizes (mm -> voxels)
    int nsx, nsy, nsz;
    int ref, n_phases;
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
