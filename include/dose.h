/*
 * dose.h -- C ABI of the GB300 Monte Carlo proton dose engine (libdose).
 *
 * The engine is the hot path of the 4D-dose calculator of Pepin et al.
 * (arXiv:1809.03927): per-phase Monte Carlo dose (Sec. 2.C) of the subplans
 * that the delivery simulation (Sec. 2.B, App. A) assigns to the breathing
 * phases of a 4DCT (Sec. 2.A), and the energy/mass-transfer accumulation of
 * the phase doses onto a reference phase (Sec. 2.D.2, Eqs. 2, 4-6).
 *
 * Conventions shared by every call
 * --------------------------------
 * Return value   DOSE_OK (0) or a negative dose_status.  Nothing is thrown
 *                across the ABI.  dose_last_error(ctx) describes the last
 *                failure on that context (dose_last_error(NULL): the last
 *                failure of a call that had no context yet, per thread).
 * Pointers       plain host or device pointers; every `*_on_device` flag
 *                says which (0: host memory, 1: device memory of the
 *                context's GPU).  Inputs are borrowed for the duration of
 *                the call only: the library copies what it keeps.
 * Ownership      a dose_ctx owns every device buffer it creates (HU grids,
 *                densities, plan, subplans, tallies, doses, accumulation
 *                buffers) and frees them in dose_destroy.
 * Streams        `stream` is a cudaStream_t passed as void* (NULL = the
 *                legacy default stream).  Calls enqueue their work on it and
 *                return without waiting, except dose_read into host memory,
 *                which waits for the stream (bounded by DOSE_OPT_TIMEOUT_MS).
 * Layout         3D grids are x fastest: index = (k * ny + j) * nx + i.  A
 *                voxel (i, j, k) covers [i dx, (i+1) dx) x [j dy, (j+1) dy) x
 *                [k dz, (k+1) dz) in grid millimetres; `origin_mm` is the
 *                patient-frame position of the grid corner.  Multi-phase
 *                arrays are phase-major: phase p starts at p * nvox.
 * Threading      a context and the contexts viewing its grid must not be
 *                used from two host threads or two streams at the same time.
 * Determinism    every history draws from a counter-based Philox4x32-10
 *                stream keyed by (seed, history index, phase); tallies are
 *                64-bit integers, so results are bit-identical run to run,
 *                for any launch shape and any batching of histories.
 */
#ifndef DOSE_H
#define DOSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dose_ctx dose_ctx;              /* opaque, owned by the library */

typedef enum dose_status {
    DOSE_OK = 0,
    DOSE_EINVAL = -1,       /* bad argument; nothing was enqueued          */
    DOSE_ENOMEM = -2,       /* device or host allocation failed            */
    DOSE_ECUDA = -3,        /* CUDA runtime error (no device, launch, ...) */
    DOSE_ETIMEOUT = -4,     /* a wait exceeded DOSE_OPT_TIMEOUT_MS         */
    DOSE_ESTEPLIMIT = -5,   /* a history hit the step cap (read back)      */
    DOSE_ESTATE = -6        /* call out of order (e.g. run before spots)   */
} dose_status;

/* One plan spot (Sec. 1 and 2.A: position, energy and weight).  x_mm, y_mm
 * are patient-frame coordinates on the two axes other than the beam axis,
 * lower axis first (beam along z: x, y; along y: x, z; along x: y, z).
 * sigma_mm is the Gaussian spot size on the entry plane.  Spots of one
 * field are delivered in array order; a layer is a maximal run of equal
 * `layer` values within the field's spots.  32 bytes.                     */
typedef struct dose_spot {
    float x_mm, y_mm, energy_MeV, sigma_mm;
    uint64_t protons;
    int32_t layer, field;
} dose_spot;

/* Delivery-clock inputs of the beam-delivery simulation (Sec. 2.B, App. A),
 * integer nanoseconds.
 * Breathing: start_phase < 0 draws the start phase of field f as word 0 of
 * Philox4x32-10(counter (f,0,0,0), key seed) mod n_phases.  Cycle c of the
 * breathing lasts n_phases t_c, t_c = floor(T_c / n_phases), with T_c =
 * period_ns, or, when period_sigma_ns > 0 (irregular breathing, one draw
 * per cycle), max(n_phases, period_ns + round(period_sigma_ns Z_c)) where
 * Z_c is the Irwin-Hall sum of the twelve 21-bit uniforms of Philox blocks
 * (f, c, 1, 0) and (f, c, 2, 0) minus 6 -- exact integers.
 * Spills: a spot's spill lasts protons * 1e9 / rate_protons_per_s ns; a
 * spill crossing a phase boundary is split by time share (floor per
 * portion, remainder to the last).  Each layer (a maximal run of equal
 * `layer` values within a field) is painted `repaints` times (floor(p/R)
 * per painting, the remainder in the last) or, if max_protons_per_paint =
 * m > 0 (then repaints must be 1), until done with min(left, m) per spot
 * and painting (isolayered repainting with a maximum per spot delivery).
 * synchrotron = 0: switch times precede every spill but a field's first
 * (layer_switch_ns before a layer's first spill, spot_switch_ns otherwise);
 * gated delivery (gated != 0) beams only in phases gate_first..gate_last
 * and at a gate-off skips to the next gate_first phase start and adds
 * discard_ns.
 * synchrotron = 1 (App. A): protons come in fills.  A fill starts with a
 * reset of layer_switch_ns (not for a field's first fill), a hold until the
 * gate is on (gated) and the beam discard of discard_ns; every layer takes a
 * new fill; a fill holds fill_protons (0: unlimited) and extracts for at
 * most extraction_limit_ns after its extraction starts (0: unlimited);
 * spills of a fill are separated by spot_switch_ns.  A spill stops at the
 * fill's charge, its time limit (then floor(w elapsed / duration) protons)
 * or a gate-off, and the rest follows at the next extraction start (a hold
 * and discard after a gate-off, a new fill otherwise).
 * Parameters must let every fill and gate window deliver a proton
 * (period_ns - 6 period_sigma_ns >= n_phases; discard shorter than the
 * gate window; with synchrotron, window - discard and extraction_limit_ns
 * at least one proton's spill time).                                      */
typedef struct dose_delivery {
    int32_t n_phases, start_phase, gated, gate_first, gate_last, repaints;
    int64_t period_ns, period_sigma_ns, spot_switch_ns, layer_switch_ns, discard_ns;
    uint64_t rate_protons_per_s, seed;
    int32_t synchrotron, reserved;
    uint64_t fill_protons;
    int64_t extraction_limit_ns;
    uint64_t max_protons_per_paint;
} dose_delivery;

/* Spread of the delivery over uncertainty trials (Sec. 2.B: start phase,
 * breathing period and synchrotron parameters varied together over 25
 * trials).  Trial k draws, under key `seed` of the mean delivery, the
 * period from {period_min_ns, + period_step_ns, ..., period_max_ns} (word 0
 * of Philox block (k,0,3,0) mod the set size; used when max > min) and each
 * synchrotron parameter j (0 spot switch, 1 layer switch, 2 discard, 3 rate,
 * 4 fill protons, 5 extraction limit) from N(mean, sigma_j) (Irwin-Hall of
 * blocks (k,j,4,0), (k,j,5,0); round half up; clamped at 0, the rate at 1;
 * sigma_j = 0 keeps the mean; sigma_j <= 2^38).  The trial's own seed,
 * which draws its start phases and breathing cycles, is seed + k *
 * 0x9E3779B97F4A7C15 (mod 2^64).                                         */
typedef struct dose_delivery_spread {
    int64_t period_min_ns, period_max_ns, period_step_ns;
    int64_t spot_switch_sigma_ns, layer_switch_sigma_ns, discard_sigma_ns;
    int64_t rate_sigma, fill_protons_sigma, extraction_limit_sigma_ns;
} dose_delivery_spread;

/* dose_read selectors */
enum {
    DOSE_PHASE_DOSE = 0,     /* float32[nvox]  Gy, phase `phase`                    */
    DOSE_DENSITY = 1,        /* float32[nvox]  g/cm^3 of phase `phase`              */
    DOSE_ACCUM = 2,          /* float32[nvox]  Gy, accumulated on the ref phase     */
    DOSE_TALLY_I64 = 3,      /* uint64[nvox]   energy in units of 2^-24 MeV x history
                                weight (weight = spot protons / its histories / (W/N)) */
    DOSE_SUBPLAN = 4,        /* uint64[n_phases * n_spots]  protons per phase, spot */
    DOSE_ENERGY_LEDGER = 5,  /* uint64[8] of phase `phase`: deposited, escaped,
                                removed, incident (2^-24 MeV units), steps,
                                histories, status flags, W (protons of the phase) */
    DOSE_STATUS = 6,         /* int32[1]: DOSE_OK or DOSE_ESTEPLIMIT for `phase`     */
    DOSE_START_PHASE = 7,    /* int32[n_fields]  start phase of each field          */
    DOSE_FIELD_END_NS = 8,   /* int64[n_fields]  delivery clock at each field's end */
    DOSE_EMTM_STATS = 9,     /* uint64[4]: subvoxels pushed (of the source voxels
                                within reach of dose), dropped (mapped outside),
                                atomic pairs issued, reserved                       */
    DOSE_HIST_PREFIX = 10,   /* uint64[n_spots + 1] of phase `phase`: first history of
                                each spot (histories of spot s = p[s+1] - p[s])      */
    DOSE_DELIVERY = 11       /* dose_delivery: the delivery the timeline ran (a
                                trial's sampled one after dose_add_spots_trials)    */
};

/* Physics switches (dose_set_option DOSE_OPT_PHYSICS), all on by default. */
enum { DOSE_PHYS_STRAGGLING = 1, DOSE_PHYS_MCS = 2, DOSE_PHYS_NUCLEAR = 4, DOSE_PHYS_ALL = 7 };

/* Options (dose_set_option).  Launch shape options change speed only,
 * never results.                                                           */
enum {
    DOSE_OPT_PHYSICS = 0,         /* bit mask of DOSE_PHYS_*                     */
    DOSE_OPT_MAX_STEPS = 1,       /* step cap per history (default 20000)        */
    DOSE_OPT_BLOCK = 2,           /* transport threads per block (64..1024, a
                                     multiple of 32; default 1024)              */
    DOSE_OPT_BLOCKS_PER_SM = 3,   /* transport blocks per SM (0 = occupancy max) */
    DOSE_OPT_CHUNK = 4,           /* histories a warp takes per queue pull (default 32) */
    DOSE_OPT_TIMEOUT_MS = 5,      /* host wait bound for dose_read (default 600000) */
    DOSE_OPT_FAIL_ALLOC_AFTER = 6,/* test hook: the n-th later device allocation
                                     of this context fails (-1 = off)            */
    DOSE_OPT_REGISTERS = 7,       /* transport register budget: 0 = up to 128 per
                                     thread (blocks <= 512), 1 = 64 (blocks <= 1024;
                                     default)                                     */
    DOSE_OPT_MATERIAL_GRID = 8    /* 1: the transport reads a per-voxel (density, SPR)
                                     grid (8 B per voxel per phase, built once per grid
                                     on first use) instead of HU + table (0, default);
                                     same results                                */
};

/* Create a context holding a voxel grid of `n_phases` HU volumes (Sec. 2.A:
 * one CT per breathing phase; Sec. 2.C: the dose grid is the CT grid) and
 * convert HU to mass density (Sec. 2.C) on the device.
 * hu: int16[n_phases * nx * ny * nz], host or device.  beam_dir must be a
 * unit axis vector (+-x, +-y, +-z): the beam enters through the upstream
 * face of the grid.  On failure *out is NULL and dose_last_error(NULL)
 * says why.                                                                 */
int dose_create_grid(dose_ctx **out, int nx, int ny, int nz, float dx_mm, float dy_mm,
                     float dz_mm, const float origin_mm[3], int n_phases, const int16_t *hu,
                     int hu_on_device, const float beam_dir[3], void *stream);

/* A new context that shares `base`'s grid and densities (read-only, kept
 * alive by a reference count) with its own plan, tallies and doses, so that
 * many dose requests over one resident 4DCT need one copy of the CT.        */
int dose_create_view(dose_ctx *base, dose_ctx **out);

/* Beam direction of one field of the plan (multi-field plans): the field's
 * spots enter along beam_dir (a unit grid-axis vector, like the grid's own
 * beam_dir) through the grid face it points into, and their x_mm, y_mm are
 * on that field's two lateral axes, lower axis first.  beam_dir = NULL
 * restores the grid's beam.  Applies to the loaded plan and to later ones;
 * views start with their base's settings.  The histories of a phase are
 * still allocated over all its spots together (each history keeps its
 * Philox stream), so a multi-field dose is the sum of its fields' parts.  */
int dose_set_field_beam(dose_ctx *c, int field, const float beam_dir[3]);

/* Load the plan (host array of n spots) and run the delivery simulation on
 * the device (Sec. 2.B): the per-phase subplans (protons per phase and
 * spot).  delivery = NULL puts every spot wholly on phase 0 (a static, 3D
 * delivery).  Replaces any previous plan and clears all phase results.
 * With the synchrotron model the call waits for the stream and reports a
 * delivery that stops making progress (DOSE_EINVAL).                      */
int dose_add_spots(dose_ctx *c, const dose_spot *spots, int64_t n,
                   const dose_delivery *delivery, void *stream);

/* Uncertainty trials (Sec. 2.B): load the plan into each of n_trials
 * contexts (views of one grid, typically) and run, in one launch, the
 * delivery simulation of trials first_trial .. first_trial + n_trials - 1,
 * each drawing its delivery from `mean` and `spread` as dose_delivery_spread
 * describes.  Waits for the stream; DOSE_EINVAL if a sampled delivery
 * breaks the progress conditions above (message names the trial).  The
 * per-phase subplans are then ready for dose_run_batch.                   */
int dose_add_spots_trials(dose_ctx *const *ctxs, int n_trials, const dose_spot *spots, int64_t n,
                          const dose_delivery *mean, const dose_delivery_spread *spread,
                          uint64_t first_trial, void *stream);

/* Monte Carlo dose of one phase's subplan (Sec. 2.C): allocate n_histories
 * over the spots in proportion to their protons (floor + largest remainder,
 * ties to the lower index), transport them through the phase's CT with
 * Philox streams keyed by (seed, history, phase), tally energy in 64-bit
 * fixed point and normalise to Gy.  spr_scale multiplies every stopping-
 * power ratio (range-uncertainty scenario); shift_mm (NULL = none) is a
 * patient setup displacement applied to the beam geometry.                 */
int dose_run_phase(dose_ctx *c, int phase, uint64_t n_histories, uint64_t seed,
                   float spr_scale, const float shift_mm[3], void *stream);

/* A ragged batch of transport jobs in one persistent launch.  Each job
 * runs histories [hist_begin, hist_end) of an n_histories-history run of
 * (ctx, phase); DOSE_JOB_CLEAR zeroes the job's tally and allocates its
 * histories first, DOSE_JOB_FINISH normalises the tally to dose after the
 * launch.  Jobs of 2^25 histories or more run in single-job launches of
 * their own, one after another on the stream, after the launch shared by
 * the others.  Splitting a run into slices over several batches gives the
 * same bits as one call, and so does any grouping of jobs into launches.
 * All contexts must live on the same GPU.                                 */
enum { DOSE_JOB_CLEAR = 1, DOSE_JOB_FINISH = 2 };
typedef struct dose_job {
    dose_ctx *ctx;
    int32_t phase;
    uint32_t flags;
    uint64_t n_histories;
    uint64_t hist_begin, hist_end;
    uint64_t seed;
    float spr_scale;
    float shift_mm[3];
} dose_job;
int dose_run_batch(const dose_job *jobs, int n_jobs, void *stream);

/* The whole 4D dose (Sec. 2.A): the Monte Carlo of every phase's subplan
 * (from the delivery given to dose_add_spots; Sec. 2.B-2.C) with
 * n_histories_per_phase histories each, all phases as one batch
 * (dose_run_batch: one persistent launch, or one launch per phase from
 * 2^25 histories; phases without protons get zero dose), then the
 * accumulation onto
 * ref_phase as in dose_accumulate_subvoxel (method 0, Eqs. 2, 4-6).  Phase p
 * uses Philox stream p under `seed`.  Reads the per-phase proton totals back
 * to the host (a short wait on the stream) to skip empty phases.           */
int dose_run_4d(dose_ctx *c, uint64_t n_histories_per_phase, uint64_t seed, float spr_scale,
                const float shift_mm[3], int ref_phase, const int nsub[3], const float *dvf,
                int dvf_on_device, const uint8_t *mask, int mask_on_device, void *stream);

/* ---- Serving: continuous batching of dose requests ---------------------
 * Requests are robust scenarios of one plan over the resident 4DCT of
 * `base` (the multiple runs of Sec. 4.C and the robust optimisation of
 * Sec. 4.C/5 need many such doses): seed, total histories (split evenly
 * over the phases the plan reaches), stopping-power scale and setup shift.
 * dose_server_step admits queued requests into free slots -- each slot is a
 * view of the base grid with the plan loaded once, created while
 * memory_budget_bytes allows and then reused -- gives every active request
 * an equal share of step_histories (at least min_slice per phase), runs all
 * those slices in one persistent launch, finishes the requests whose last
 * slice ran (normalisation, and the accumulation onto ref_phase when
 * `accumulate`; dvf is a device array as in dose_accumulate_subvoxel) and
 * waits for the stream.  A request's result is bit-identical to the same
 * request served alone: histories are keyed by (seed, history, phase).
 * dose_server_create runs the delivery timeline of the plan once, on a
 * template view of `base`; slots copy that plan, its subplan and its field
 * beams, so field beams set on the base later do not reach the server
 * (launch options are read from the base when a slot is created).         */
typedef struct dose_server dose_server;
typedef struct dose_server_config {
    uint64_t memory_budget_bytes;
    uint64_t step_histories;
    uint64_t min_slice;
    int32_t max_active;        /* 0: no cap beyond the budget */
    int32_t ref_phase;
    int32_t nsub[3];
    int32_t accumulate;
    const float *dvf;          /* device, n_phases x 3 x nvox mm, or NULL = identity */
    int32_t policy;            /* DOSE_SERVE_FAIR or DOSE_SERVE_SHORTEST_FIRST */
    int32_t max_wait_steps;    /* shortest-first: bound on the steps in a row a request goes
                                  without a slice (0: none) */
} dose_server_config;
/* How a step's histories are shared among the active requests: equally
 * (each at least min_slice per phase), or to the requests with the fewest
 * histories left first (the step's budget handed out in that order; a
 * request without a slice waits), which shortens the small requests'
 * latency without stretching the large ones as much as equal shares do.
 * Under a sustained overload shortest-first alone can hold a large request
 * back indefinitely; with max_wait_steps = k > 0 a request that has gone k
 * steps in a row without a slice is served first at the next step, with
 * at least min_slice histories per phase even when the step's budget is
 * spent, so no request waits more than k steps in a row.                  */
enum { DOSE_SERVE_FAIR = 0, DOSE_SERVE_SHORTEST_FIRST = 1 };
typedef struct dose_request {
    uint64_t n_histories;
    uint64_t seed;
    float spr_scale;
    float shift_mm[3];
    /* the request's own delivery (a gating or repainting variant, Sec. 2.B),
     * copied at submission; NULL = the server's.  A request whose delivery
     * puts no protons on any phase finishes with zero dose.               */
    const dose_delivery *delivery;
} dose_request;
int dose_server_create(dose_ctx *base, const dose_server_config *cfg, const dose_spot *spots,
                       int64_t n_spots, const dose_delivery *delivery, dose_server **out);
int dose_server_submit(dose_server *s, const dose_request *req, int64_t *id);
/* completed (host, max_completed entries) receives the ids finished by this step. */
int dose_server_step(dose_server *s, void *stream, int64_t *completed, int max_completed,
                     int *n_completed);
/* Read a finished request's result (selectors as dose_read); valid until
 * dose_server_release frees its slot.                                      */
int dose_server_result(dose_server *s, int64_t id, int what, int phase, void *dst, size_t bytes,
                       int dst_on_device, void *stream);
int dose_server_release(dose_server *s, int64_t id);
/* out: queued, active, slots, completed, histories run, steps, bytes per
 * slot, finished but not released.                                         */
int dose_server_stats(const dose_server *s, uint64_t out[8]);
/* Where the served time went, summed over all steps so far (seconds): out[0]
 * device time of the steps' transport batches (history allocation,
 * transport, normalisation; CUDA events on the step's stream), out[1]
 * device time of the finishing requests' accumulations (zero phases, EMTM,
 * Eq. 2), out[2] host wall time of the steps (admission, job building,
 * launches and the wait), out[3] steps that ran a batch.                  */
int dose_server_timing(const dose_server *s, double out[4]);
void dose_server_destroy(dose_server *s);

/* Supply the dose of one phase from outside (float32[nvox] Gy), e.g. to
 * accumulate doses computed elsewhere.                                     */
int dose_set_phase_dose(dose_ctx *c, int phase, const float *dose, int dose_on_device,
                        void *stream);

/* A deformable registration's vector grid as DICOM stores it (App. B):
 * N_X x N_Y x N_Z grid voxels, the patient-frame centre of voxel (0,0,0),
 * the spacings dX, dY, dZ, the row (U) and column (V) direction cosines
 * (orthonormal; the depth direction is W = U x V) and the rigid transforms
 * applied before and after the deformation (row-major 4 x 4; the identity
 * between 4DCT phases).                                                   */
typedef struct dose_dvf_grid {
    int32_t n[3];
    float start_mm[3];
    float spacing_mm[3];
    float row_cos[3];
    float col_cos[3];
    float pre[16];
    float post[16];
} dose_dvf_grid;

/* Decode a registration onto this context's CT grid (App. B, Eqs. 7-8):
 * grid voxel (i, j, k) sits at r0 = start + i dX U + j dY V + k dZ W
 * (Eq. 8) and maps to r_f = M_post (M_pre r0 + Delta_ijk) (Eq. 7); a point
 * between grid voxels maps to the trilinear interpolant of the r_f around
 * it (the DICOM rule the paper quotes).  Every CT voxel centre p = origin +
 * (i + 1/2) d inside the hull of grid voxel centres gets the displacement
 * r_f(p) - p in dvf_out; outside it gets 0, and mask_inout (if not NULL) is
 * cleared there, so decoding every phase's registration into one mask
 * leaves the region all of them cover (the report mask of Sec. 2.D.2).
 * translation: float32[N_Z][N_Y][N_X][3] mm (x fastest, components
 * interleaved), host or device.  dvf_out: device float32[3 * nvox] (x, y,
 * z component planes: one phase's block of the dvf argument below).
 * mask_inout: device uint8[nvox] or NULL.  The inside test is taken in
 * single precision in a fixed order, so it is reproducible bit for bit.
 * Errors: DOSE_EINVAL for a non-positive size or spacing, direction cosines
 * that are not orthonormal (1e-4) or outputs that are not device memory.  */
int dose_decode_dvf(dose_ctx *c, const dose_dvf_grid *grid, const float *translation,
                    int translation_on_device, float *dvf_out, uint8_t *mask_inout, void *stream);

/* Accumulate the phase doses onto ref_phase (Sec. 2.D.2).  method 0 is the
 * energy/mass-transfer method of Eqs. 4-6: every voxel of each source phase
 * S != ref_phase is split into nsub[0] x nsub[1] x nsub[2] subvoxels whose
 * centres move by S's DVF (trilinear between voxel centres, clamped at the
 * edges) into the reference voxel whose half-open cell holds them; subvoxel
 * mass rho_j v_k and energy rho_j v_k D_j are summed per reference voxel in
 * 64-bit fixed point, D_i^S = sum E / sum M (0 where nothing lands), and
 * D_i = D_i^R + sum_S D_i^S (Eq. 2), zero where mask == 0.
 * dvf: float32[n_phases * 3 * nvox] mm, the displacement carrying a point
 * of phase S to the reference (component-major per phase); NULL = identity.
 * mask: uint8[nvox] or NULL (all ones).
 * method 1 is the dose-interpolation method of Eq. 3: every voxel i of the
 * reference phase is split into nsub subvoxels whose centres are carried to
 * each source phase S by the reference-to-S displacement, the dose of S is
 * interpolated trilinearly (between voxel centres, clamped at the edges) at
 * each carried point, and D_i^S is the mean over the subvoxels; then Eq. 2
 * and the mask as above.  For method 1, dvf holds for each phase S the
 * displacement (mm) carrying a reference point to S, given at the reference
 * voxel centres -- the opposite direction to method 0, as the paper notes.
 * Every phase must have a dose.  DOSE_EMTM_STATS is only readable after
 * method 0.
 * Both methods visit only what a phase's dose can reach: the box of the
 * voxels carrying dose (method 0: rho > 0 and D > 0; method 1: D != 0),
 * grown per axis by m (ceil(max|u| / d) + 2) voxels, u the phase's field,
 * m = 2 for method 0 (source voxels) and 1 for method 1 (reference voxels).
 * What lies outside adds exactly zero, so the result is that of visiting
 * every voxel; DOSE_EMTM_STATS counts the subvoxels within reach.          */
int dose_accumulate_subvoxel(dose_ctx *c, int ref_phase, const int nsub[3], const float *dvf,
                             int dvf_on_device, const uint8_t *mask, int mask_on_device,
                             int method, void *stream);

/* Copy a result (see the selectors) into dst (`bytes` must equal its size).
 * Into host memory the call waits for `stream`; into device memory it only
 * enqueues the copy.                                                       */
int dose_read(dose_ctx *c, int what, int phase, void *dst, size_t bytes, int dst_on_device,
              void *stream);

/* Autotuner: time the transport of histories [0, sample_histories) of an
 * n_histories-history run of `phase` under each launch shape -- register
 * budget (DOSE_OPT_REGISTERS 0 or 1) x threads per block in {128, 256, 512,
 * 1024} (the shapes that fit) x histories a warp takes per queue pull in
 * {32, 64, 128, 256} -- then, for the fastest, the material source
 * (DOSE_OPT_MATERIAL_GRID 0 or 1, each timed twice, the faster minimum
 * kept), and keep the winners on the context.
 * Launch shapes change speed only: the tallies are bit-identical.  The
 * phase's tally and dose are overwritten.  best (host, may be NULL)
 * receives {registers option, block, chunk, elapsed microseconds of the best
 * shape}.  Waits for the stream.  The step-length rule is part of the
 * physics model and is not tuned.                                          */
int dose_autotune(dose_ctx *c, int phase, uint64_t n_histories, uint64_t sample_histories,
                  uint64_t seed, void *stream, int64_t best[4]);

/* Autotuner for a ragged batch (the launch dose_run_batch makes of `jobs`):
 * times a sample of about sample_histories histories spread over the jobs
 * in proportion to their ranges (job k: the first histories of its range)
 * under the launch shapes and material sources of dose_autotune, with the
 * kernel the batch itself launches, and sets the winners on every context
 * of the batch.  Every (context, phase) of the batch is cleared and its
 * histories allocated first; their tallies and doses are overwritten, so
 * run the batch (with DOSE_JOB_CLEAR) afterwards.  best as dose_autotune.
 * Waits for the stream.                                                    */
int dose_autotune_batch(const dose_job *jobs, int n_jobs, uint64_t sample_histories, void *stream,
                        int64_t best[4]);

/* Set an option (DOSE_OPT_*).                                              */
int dose_set_option(dose_ctx *c, int option, int64_t value);

/* Read an option's current value (e.g. the launch shape the autotuner
 * kept).  value: host pointer.  DOSE_EINVAL for an unknown option.        */
int dose_get_option(const dose_ctx *c, int option, int64_t *value);

/* Free the context (waits for its device work).  NULL is a no-op.          */
void dose_destroy(dose_ctx *c);

/* Text of the last failure on c (or of this thread's last context-less
 * failure when c is NULL).  Valid until the next call on c.               */
const char *dose_last_error(const dose_ctx *c);

/* Library version, for the binding's load check.                           */
int dose_version(void);

/* Dose of one static plan without allocating device memory.
 *
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc -- code inside a framework or service that owns the device's
 * memory through its own allocator, or that must not allocate once it is
 * running.  The caller passes device input and output buffers; every other
 * buffer the kernels use (tally, spot table, history allocation, ledger,
 * work counter, allocation descriptor, lookup tables) lives in one
 * fixed-size static device array that each GPU loading this library holds
 * until the process exits.  No cudaMalloc, cudaFree or allocating library
 * routine is called.
 *
 * Computes what dose_create_grid + dose_add_spots(delivery NULL) +
 * dose_run_phase(phase 0, spr_scale 1, no shift) compute with the default
 * options, bit for bit: hu is int16[nx*ny*nz] in device memory (x fastest)
 * on the current device, spots is a host array whose spots all belong to
 * field 0, dose receives float32[nx*ny*nz] Gy in device memory on the
 * current device; ledger_out (host, may be NULL) receives the 8-word ledger
 * of DOSE_ENERGY_LEDGER.  The call works on `stream` (NULL: the legacy
 * default stream) and returns once the dose is written: it waits for the
 * stream.  Returns DOSE_ESTEPLIMIT (dose and ledger written) when a history
 * reached the step limit.
 * Limits: nx*ny*nz <= DOSE_NOALLOC_MAX_VOXELS and n_spots <=
 * DOSE_NOALLOC_MAX_SPOTS; larger inputs, a non-finite origin or a spot of
 * another field return DOSE_EINVAL with a message in dose_last_error(NULL).
 * The pointers are not checked (the caller guarantees their sizes, types
 * and device).
 * The first call on a device sets the array up for that device (finds its
 * device address, uploads the tables) and waits for it: make that first
 * call before any stream capture.  All calls share the one array, which
 * keeps the previous call's contents (the call clears what must start at
 * zero): calls from several host threads at once race on it and must be
 * serialised by the caller.                                                */
#define DOSE_NOALLOC_MAX_VOXELS 2097152   /* 2^21, e.g. 128^3: 16 MiB of tally */
#define DOSE_NOALLOC_MAX_SPOTS 4096
int dose_run_phase_noalloc(const int16_t *hu, int nx, int ny, int nz, float dx_mm, float dy_mm,
                           float dz_mm, const float origin_mm[3], const float beam_dir[3],
                           const dose_spot *spots, int n_spots, uint64_t n_histories, uint64_t seed,
                           float *dose, uint64_t ledger_out[8], void *stream);

/* Measured throughput peaks of the current device, for the roofline of the
 * transport (Sec. 2.C engine; the paper has no such call): out[0] = issue
 * rate of a mixed FP32/INT32 instruction stream (8 FFMA, 4 IMAD, 4 LOP3 per
 * 16 instructions on independent chains, 64 warps per SM), thread
 * instructions per second; out[1] = the same for FFMA alone; out[2] =
 * 64-bit atomic additions per second to pseudo-random elements of a
 * 16.8 MB array (L2-resident, like the dose tally); out[3] = the SM count.
 * Each rate is the best of three timings of a fixed workload of a few
 * milliseconds on `stream`; the call allocates and frees its 16.8 MB
 * scratch and waits for the stream.  DOSE_ECUDA on a CUDA error.           */
int dose_measure_peaks(double out[4], void *stream);

/* Self-test of the device random-number generator: Philox4x32-10 (Salmon
 * et al., SC'11; the generator of Sec. 2.B, footnote b) of n counters
 * ctr[4 i..4 i+3] under keys key[2 i..2 i+1] into out[4 i..], and the six
 * 21-bit uniforms (k + 1/2) 2^-21 the transport draws from each block into
 * uniforms[6 i..] (NULL: skipped).  All pointers are host memory; the call
 * runs on the current device and waits for it.                              */
int dose_debug_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n,
                      float *uniforms);

/* Self-test of the device lookup tables: for each of the n energies E[i]
 * (host, MeV) writes out[5 i..5 i+4] = CSDA range R(E) in mm of water, the
 * energy at that range E(R(E)), the Bohr variance per mm of water path, the
 * Highland coefficient (13.6/pv)^2 and the nuclear Sigma per mm, each
 * evaluated exactly as the transport does.  Host memory; waits.            */
int dose_debug_tables(const float *E, int n, float *out, void *stream);

/* Self-test of the birth order of a job's histories (no device work): for
 * work items w = 0 .. n-1 writes out[w] = the history index (from the
 * job's first) that work item w transports: the last t = min(n/8, 2^18)
 * work items take the last t histories in order, the others are dealt
 * round-robin over 2^log2_strides contiguous strides of the first n - t
 * histories (the order the transport uses for large jobs on grids small
 * enough for the L2; 0 is plan order).  A history's result depends only on
 * its index, so the order changes no tally.  n <= 2^26, log2_strides <= 16;
 * host memory.                                                            */
int dose_debug_spread(uint64_t n, uint32_t log2_strides, uint64_t *out);

#ifdef __cplusplus
}
#endif
#endif /* DOSE_H */
