// Internal definitions of the CUDA dose engine: model constants, lookup-
// table layout, per-launch job descriptors and small device helpers.
// Included by the engine's translation units only.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace dose {

// ---- transport model (project choices; the paper prints no physics) -----
constexpr float kEcut = 0.5f;          // MeV: below this the rest is deposited
constexpr float kFstep = 0.25f;        // step <= 0.25 x residual range in the medium
constexpr float kSmin = 0.01f;         // mm, shortest physics step
constexpr float kFloc = 0.6f;          // local fraction at nuclear removal
constexpr float kInvX0 = 1.0f / 360.8f;// 1/(water radiation length, mm at 1 g/cm^3)
constexpr float kHighlandB = 0.038f;
constexpr float kInvSqrt12 = 0.28867513459481287f;
constexpr float kQuantum = 16777216.0f;   // tally units per MeV (2^24)

// ---- lookup tables (built in FP64 on the host, stored FP32) -------------
// re, hs: uniform kinetic-energy grid E_i = i * kDE, i = 0..kNE.
// er:     grid uniform in sqrt(range): R_i = (i * kDS)^2, i = 0..kNR.
// mat:    HU -1000..3000 -> (rho g/cm^3, SPR).
constexpr int kNE = 2048;
constexpr float kEmax = 256.0f;
constexpr float kDE = kEmax / kNE;
constexpr float kInvDE = kNE / kEmax;
constexpr int kNR = 2048;
constexpr float kRmax = 420.0f;        // mm, above the range of 256 MeV
constexpr int kHuMin = -1000, kHuMax = 3000, kNHU = kHuMax - kHuMin + 1;

// Each entry of re, hs and er also holds its FP32 difference to the next
// entry (d = next - this, rounded as the FP32 subtraction rounds it), so a
// lookup is one load and fma(f, d, value).
struct Tables {
    float4 re[kNE + 2];   // (CSDA range in water, mm; Bohr variance per mm of water path, MeV^2/mm; d, d)
    float4 hs[kNE + 2];   // (p v in MeV, for the Highland coefficient; nuclear Sigma per mm of water; d, d)
    float2 er[kNR + 4];   // (energy at range (i kDS)^2; d)
    float2 mat[kNHU + 3]; // (rho, SPR)
};
static_assert(sizeof(Tables) % 16 == 0, "tables are copied to shared memory as int4");
// The transport stages the physics tables (re, hs, er) in shared memory and
// reads the HU table through the L1 cache.
constexpr size_t kSmemTables = offsetof(Tables, mat);
static_assert(kSmemTables % 16 == 0, "staged part must be a multiple of 16 bytes");

// Host-side FP64 builder (lut.cpp).  inv_ds receives 1/kDS.
void build_tables(Tables *t, float *inv_ds);

// ---- ledger words per phase/job ------------------------------------------
enum { LED_DEP = 0, LED_ESC = 1, LED_REM = 2, LED_INC = 3, LED_STEPS = 4, LED_HIST = 5,
       LED_FLAGS = 6, LED_W = 7, LED_WORDS = 8 };
enum { FLAG_STEPLIMIT = 1 };

// ---- one transport job of a persistent launch ---------------------------
struct alignas(16) TJob {
    // read every step, grouped in 16-byte words for vector loads
    int nx, ny, nz;
    unsigned max_steps;
    float dx, dy, dz;
    float spr_scale;
    float idx, idy, idz;                // 1 / voxel sizes
    unsigned physics;
    uint4 rk[5];                        // Philox round keys: (k0, k1) of rounds 2i and 2i+1
    const int16_t *hu;                  // this phase's grid
    const float2 *matg;                 // this phase's (rho, SPR) per voxel, or null: hu + table
    unsigned long long *tally;          // nvox
    unsigned long long *ledger;         // LED_WORDS
    // read at history birth
    const float4 *spot;                 // (x, y, E, sigma) patient mm / MeV
    const float *wh;                    // history weight per spot
    const unsigned long long *prefix;   // n_spots + 1 (first history of each spot)
    const unsigned char *spot_dir;      // per spot: 2 axis + (sign > 0), or null: beam_axis/sign
    int n_spots;
    float o[3];                         // patient->grid offsets per axis (origin + shift)
    int beam_axis, beam_sign;
    unsigned key0, key1, stream;
    unsigned spread_log2;               // work items spread over 2^spread_log2 strides (see spread_history)
    unsigned long long hist_begin;      // first history of this slice
    unsigned long long work_begin;      // offset in the launch's work index
    unsigned long long n_work;          // work items (histories) of this slice
};
static_assert(sizeof(TJob) == 256, "job descriptor: 256 bytes");

// The order in which a job's histories are born: work item w of n goes to
// history spread_history(w, n, s), a bijection of [0, n).  The last
// t = min(n / 8, 2^18) work items take the last t histories in plan order;
// the others are dealt round-robin over 2^s contiguous strides of the first
// n - t histories (stride k holds (n - t) / 2^s of them, one more for the
// first (n - t) mod 2^s).  Consecutive work items, and so the histories in
// flight, then come from 2^s places of the plan instead of a few
// neighbouring spots, whose tracks would overlap and pile their tally
// atomics onto the same voxels; the launch still ends on the plan's last
// (lowest-energy, shortest) spots, which keeps its tail short.  A
// history's result depends only on its index, so the order changes no
// tally bit.  s = 0 is the identity.
constexpr unsigned kSpreadTailLog2 = 18;
__host__ __device__ inline unsigned long long spread_history(unsigned long long w, unsigned long long n, unsigned s)
{
    const unsigned long long t = (n >> 3) < (1ull << kSpreadTailLog2) ? (n >> 3) : (1ull << kSpreadTailLog2);
    if (s == 0 || w >= n - t) return w;
    const unsigned long long ns = n - t, m = (1ull << s) - 1, q = ns >> s, r = ns & m, k = w & m;
    return k * q + (k < r ? k : r) + (w >> s);
}
// Jobs of at least kSpreadMinWork histories on grids whose tally and
// material grid (16 bytes a voxel) fit kSpreadGridBytes of the L2 take 64
// strides.  Larger grids keep plan order, whose few neighbouring spots keep
// the L2 working set small; so do smaller jobs, whose launch tail grows
// when the last histories in flight mix all energies instead of ending on
// the plan's last, lowest-energy spots.
constexpr unsigned kSpreadLog2 = 6;
constexpr unsigned long long kSpreadGridBytes = 48ull << 20;
constexpr unsigned long long kSpreadMinWork = 1ull << 23;
inline unsigned spread_for(long long nvox, unsigned long long n_work)
{
    return (unsigned long long)nvox * 16 <= kSpreadGridBytes && n_work >= kSpreadMinWork ? kSpreadLog2 : 0;
}

// The fields every step reads that jobs of one context and seed share;
// they precede the per-job pointers (no padding: all 4-byte scalars and
// 16-byte vectors).
constexpr size_t kStepFieldBytes = offsetof(TJob, hu);
static_assert(kStepFieldBytes == 128, "per-step shared fields: 12 words and five round-key words");

// A transport launch's dynamic shared memory holds the physics tables, the
// warps' birth buffers (birth_smem(block)) and, when staged, the descriptors
// and per-job counters (escaped, removed, steps, flags) of up to
// kMaxStagedJobs jobs: transport_smem(n) + birth_smem(block).  The launcher
// stages only where that costs no resident blocks, else passes
// transport_smem(kMaxStagedJobs + 1) + birth_smem(block) (no jobs) and the
// kernel reads the jobs from global memory.
constexpr int kMaxStagedJobs = 256;
static_assert(sizeof(TJob) % 8 == 0, "job counters follow the descriptors 8-byte aligned");
__host__ __device__ constexpr size_t transport_smem(int n_jobs)
{
    return kSmemTables + (n_jobs <= kMaxStagedJobs ? (size_t)n_jobs * (sizeof(TJob) + 4 * sizeof(unsigned long long)) : 0);
}
constexpr size_t kSmemTransportMax = transport_smem(kMaxStagedJobs);
// Staging stops where it would leave the block's SM less than ~75 KB of L1
// for the grid and HU-table reads: a 243-job trial batch staged at 1024
// threads (213 KB of shared memory) ran at 2.0e8 histories/s instead of
// 2.7e8 unstaged, while a 74-job batch (169 KB) gains 3.5 % from staging.
constexpr size_t kStageSmemCap = 180 * 1024;
// Per warp, a buffer of 32 born histories between the tables and the staged
// jobs: kBirthWords planes (position, direction, energy, nuclear path, weight,
// voxel, job, history index) of 32 slots per warp.
constexpr int kBirthWords = 15;
__host__ __device__ constexpr size_t birth_smem(int block)
{
    return (size_t)(block / 32) * 32 * kBirthWords * sizeof(float);
}

struct AllocJob {
    const unsigned long long *protons;  // n_spots, this phase's subplan
    const float4 *spot;                 // (x, y, E, sigma): energies for the incident total
    unsigned long long *rem;            // scratch n_spots
    unsigned long long *prefix;         // n_spots + 1
    float *wh;                          // n_spots
    unsigned long long *ledger;         // LED_W receives W
    int n_spots;
    unsigned long long n_hist;
};

struct NormJob {
    const unsigned long long *tally;
    unsigned long long *ledger;         // reads LED_W, adds the tally sum to LED_DEP
    const float *rho;
    float *dose;
    unsigned long long n_hist;
    double voxel_cm3;
    long long nvox;
};

#if defined(__CUDACC__)
// ---- Philox4x32-10 (Salmon et al., SC'11) -------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned k0, unsigned k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Philox4x32-10 with the ten round keys given (the key schedule of the
// definition, precomputed per job, two rounds per 16-byte word).
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint4 *rk)
{
#pragma unroll
    for (int r = 0; r < 10; r += 2) {
        const uint4 k = rk[r >> 1];
        unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        hi0 = __umulhi(0xD2511F53u, c.x); lo0 = 0xD2511F53u * c.x;
        hi1 = __umulhi(0xCD9E8D57u, c.z); lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.z, lo1, hi0 ^ c.w ^ k.w, lo0);
    }
    return c;
}

// Six 21-bit uniforms (k + 1/2) 2^-21 from the 128 bits of a block, bits
// [21 i, 21 i + 21) of the little-endian word concatenation.  Each value is
// assembled exactly: k goes into the top of the mantissa of 1.0f with the
// half-unit bit set, which reads 1 + (k + 1/2) 2^-21, and 1 is subtracted
// (exact: the difference has at most 22 significant bits).
struct U6 { float u[6]; };
__device__ __forceinline__ float unit_from_bits(unsigned b)   // k in bits [2, 23)
{
    return __int_as_float((b & 0x007FFFFCu) | 0x3F800002u) - 1.0f;
}
__device__ __forceinline__ float one_plus_unit(unsigned b)    // 1 + (k + 1/2) 2^-21, k in bits [2, 23)
{
    return __int_as_float((b & 0x007FFFFCu) | 0x3F800002u);
}
__device__ __forceinline__ U6 uniforms6(uint4 w)
{
    // the six subtractions of 1 as three paired additions (exact either way)
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 a = __fadd2_rn(make_float2(one_plus_unit(w.x << 2),                        // bits 0..20
                                            one_plus_unit(__funnelshift_r(w.x, w.y, 19))), m1);   // 21..41
    const float2 b = __fadd2_rn(make_float2(one_plus_unit(w.y >> 8),                        // bits 42..62
                                            one_plus_unit(__funnelshift_r(w.y, w.z, 29))), m1);   // 63..83
    const float2 c = __fadd2_rn(make_float2(one_plus_unit(__funnelshift_r(w.z, w.w, 18)),   // 84..104
                                            one_plus_unit(w.w >> 7)), m1);                        // 105..125
    U6 r;
    r.u[0] = a.x; r.u[1] = a.y; r.u[2] = b.x; r.u[3] = b.y; r.u[4] = c.x; r.u[5] = c.y;
    return r;
}

// Square root through the hardware reciprocal square root (x >= 0).
__device__ __forceinline__ float fast_sqrt(float x)
{
    return x > 0.0f ? x * rsqrtf(x) : 0.0f;
}

// Box-Muller pair: r = sqrt(-2 ln ua), (r cos 2 pi ub, r sin 2 pi ub).  The
// angle is evaluated as 2 pi ub - pi in (-pi, pi), where the fast sine and
// cosine are accurate; cos(x + pi) = -cos x and sin(x + pi) = -sin x.
__device__ __forceinline__ float2 box_muller(float ua, float ub)
{
    // ua is in (0, 1), so t > 0; the floor only keeps rsqrt finite
    const float t = fmaxf(-2.0f * __logf(ua), 1e-30f);
    const float r = t * rsqrtf(t);
    const float a = __fmaf_rn(6.28318530717958647f, ub, -3.14159265358979324f);
    float s, c;
    __sincosf(a, &s, &c);
    return make_float2(-r * c, -r * s);
}

// First normal of the Box-Muller pair only.
__device__ __forceinline__ float box_muller_first(float ua, float ub)
{
    const float t = fmaxf(-2.0f * __logf(ua), 1e-30f);
    const float r = t * rsqrtf(t);
    const float a = __fmaf_rn(6.28318530717958647f, ub, -3.14159265358979324f);
    return -r * __cosf(a);
}

// Energy loss of a step whose mean (CSDA) loss is m and whose Bohr variance
// is v, from the standard normal z: lognormal with exactly that mean and
// variance, m exp(sig z - sig^2 / 2) with sig^2 = ln(1 + v / m^2), so the
// moments of the loss along a path do not depend on how it is cut into
// steps.  Evaluated in base 2 with the hardware's approximate log2 and exp2
// (PTX lg2.approx, ex2.approx): with L = log2(1 + v / m^2), the exponent
// sig z - sig^2 / 2 is (sqrt(L log2(e)) z - L / 2) ln 2.  A step without a
// positive mean loss keeps its CSDA loss (no fluctuation); m > 0 here is at
// least an FP32 unit of the energy, so m * m does not underflow.
__device__ __forceinline__ float straggle_loss(float m, float v, float z)
{
    const float x = __fdividef(v, m * m);
    float L, f;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(L) : "f"(1.0f + x));
    const float r = fast_sqrt(L * 1.44269504088896341f);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"(fmaf(r, z, -0.5f * L)));
    return m > 0.0f ? m * f : m;
}

// a / b in FP64 for b > 0 without the library's double division (slow on
// this part's FP64 units): the FP32 reciprocal refined by one Newton-Raphson
// step y <- y + y (1 - b y) (24 -> ~48 correct bits), then one residual
// correction of the quotient, q <- q + y (a - b q), which brings it within
// an ulp of the correctly rounded quotient.
__device__ __forceinline__ double div64(double a, double b)
{
    double y = (double)__frcp_rn((float)b);
    y = fma(y, fma(-b, y, 1.0), y);
    const double q = a * y;
    return fma(y, fma(-b, q, a), q);
}

__device__ __forceinline__ unsigned long long to_units(float e)
{
    return __float2ull_rn(e * kQuantum);
}

// Highland coefficient (13.6 MeV / pv)^2 from the tabulated p v.
__device__ __forceinline__ float highland_coeff(float pv)
{
    const float k = __fdividef(13.6f, pv);
    return k * k;
}

// Linear interpolation on the uniform energy grid.
__device__ __forceinline__ float2 lerp_e(const float4 *t, float e)
{
    const float x = e * kInvDE;                      // e >= 0 on every call
    const int i = (int)min((unsigned)(int)x, (unsigned)(kNE - 1));
    const float f = x - (float)i;
    const float4 a = t[i];
    return make_float2(fmaf(f, a.z, a.x), fmaf(f, a.w, a.y));
}

// Energy at a residual water range, linear on the sqrt(range) grid.
__device__ __forceinline__ float energy_at_range(const float2 *er, float r, float inv_ds)
{
    const float x = fast_sqrt(r) * inv_ds;
    const int i = (int)min((unsigned)(int)x, (unsigned)(kNR - 1));
    const float f = x - (float)i;
    const float2 a = er[i];
    return fmaf(f, a.y, a.x);
}

// The voxels an accumulation of one source phase has to visit: the box of
// the voxels that carry dose (a reach record, words as k_reach writes them)
// grown on every axis by `mult` x r voxels, r = ceil(max|u| / d) + 2, and
// clipped to the grid; empty (lo > hi) when no voxel carries dose.  A point
// carried by the field moves at most max|u| / d voxels (a trilinear blend
// of node values cannot exceed their largest magnitude; the FP32 roundings
// add far less than the one voxel of slack in r), so
//   DIM  (mult 1): a reference voxel outside the box interpolates only zero
//        dose taps of the phase;
//   EMTM (mult 2): a source voxel outside the box can push only to voxels
//        that receive no energy, whose dose is zero with or without its mass.
// A non-finite or grid-sized displacement gives the whole axis.
struct VoxBox { int lo[3], hi[3]; };
__device__ __forceinline__ VoxBox reach_box(const unsigned *w, int mult, int nx, int ny, int nz,
                                            float idx, float idy, float idz)
{
    VoxBox b;
    const int n[3] = {nx, ny, nz};
    const float id[3] = {idx, idy, idz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (w[3] == 0) { b.lo[ax] = 0; b.hi[ax] = -1; continue; }
        const float dm = __uint_as_float(w[6 + ax]) * id[ax];
        const int r = dm < (float)n[ax] ? (int)ceilf(dm) + 2 : n[ax];
        b.lo[ax] = max((int)~w[ax] - mult * r, 0);
        b.hi[ax] = min((int)w[3 + ax] - 1 + mult * r, n[ax] - 1);
    }
    return b;
}
#endif  // __CUDACC__

}  // namespace dose
