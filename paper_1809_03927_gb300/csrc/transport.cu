// Transport-side kernels of the dose engine (Sec. 2.C of Pepin et al.):
//   k_density    HU -> mass density of every voxel
//   k_alloc      histories per spot (floor + largest remainder), prefix sums,
//                history weights and the phase's proton total W
//   k_transport  persistent, warp-cooperative class II condensed-history
//                transport with a 64-bit fixed-point energy tally
//   k_normalise  tally -> dose in Gy
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include "engine.cuh"
#include "kernels.h"

namespace dose {

namespace {
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Block-wide sum; every thread gets the total.  blockDim.x % 32 == 0.
__device__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_u64(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    unsigned long long t = 0;
    for (int w = 0; w < nw; ++w) t += red[w];
    return t;
}

// Block-wide exclusive prefix sum of one value per thread.
__device__ unsigned long long block_exclusive_u64(unsigned long long v, unsigned long long *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    unsigned long long base = 0;
    for (int w = 0; w < warp && w < nw; ++w) base += red[w];
    return base + incl - v;
}

// (a b) / w and (a b) mod w for 64-bit a, b, w with a b / w < 2^64.
__device__ void mul_divmod(unsigned long long a, unsigned long long b, unsigned long long w,
                           unsigned long long *q, unsigned long long *r)
{
    const unsigned long long lo = a * b, hi = __umul64hi(a, b);
    unsigned long long rem = hi, quo = 0;
    for (int i = 63; i >= 0; --i) {
        const unsigned long long carry = rem >> 63;
        rem = (rem << 1) | ((lo >> i) & 1ull);
        quo <<= 1;
        if (carry || rem >= w) { rem -= w; quo |= 1ull; }
    }
    *q = quo;
    *r = rem;
}
}  // namespace

// ------------------------------------------------------------------ density
__global__ void k_density(const int16_t *__restrict__ hu, float *__restrict__ rho, long long n,
                          const Tables *__restrict__ tab)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int h = min(max((int)hu[i], kHuMin), kHuMax);
        rho[i] = tab->mat[h - kHuMin].x;
    }
}

// HU -> (density, SPR) of every voxel: the table's values, for launches that
// read the material per voxel instead of HU + table.
__global__ void k_material(const int16_t *__restrict__ hu, float2 *__restrict__ m, long long n,
                           const Tables *__restrict__ tab)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int h = min(max((int)hu[i], kHuMin), kHuMax);
        m[i] = tab->mat[h - kHuMin];
    }
}

// --------------------------------------------------------------- allocation
// One block per job.  n_s = floor(N p_s / W) for every spot, then the
// N - sum n_s spots with the largest remainders (ties: lower index) get one
// more; prefix[s] is the first history of spot s; wh[s] = p_s N / (n_s W).
__global__ void __launch_bounds__(1024) k_alloc(const AllocJob *__restrict__ jobs)
{
    __shared__ unsigned long long red[32];
    __shared__ unsigned long long tile[1024];
    const AllocJob J = jobs[blockIdx.x];
    const int S = J.n_spots, tid = threadIdx.x, bs = blockDim.x;
    const unsigned long long N = J.n_hist;

    unsigned long long w = 0;
    for (int s = tid; s < S; s += bs) w += J.protons[s];
    const unsigned long long W = block_sum_u64(w, red);
    if (W == 0 || N == 0) {
        for (int s = tid; s <= S; s += bs) J.prefix[s] = 0;
        for (int s = tid; s < S; s += bs) J.wh[s] = 0.0f;
        if (tid == 0) J.ledger[LED_W] = W;
        return;
    }
    unsigned long long used = 0;
    for (int s = tid; s < S; s += bs) {
        unsigned long long q, r;
        mul_divmod(N, J.protons[s], W, &q, &r);
        J.prefix[s + 1] = q;       // n_s for now
        J.rem[s] = r;
        used += q;
    }
    const unsigned long long left = N - block_sum_u64(used, red);
    __syncthreads();
    for (int base = 0; base < S; base += bs) {
        const int s = base + tid;
        const unsigned long long rs = s < S ? J.rem[s] : 0ull;
        unsigned long long rank = 0;
        for (int t0 = 0; t0 < S; t0 += 1024) {
            __syncthreads();
            for (int k = tid; k < 1024 && t0 + k < S; k += bs) tile[k] = J.rem[t0 + k];
            __syncthreads();
            const int tn = min(1024, S - t0);
            if (s < S)
                for (int k = 0; k < tn; ++k) {
                    const unsigned long long rt = tile[k];
                    rank += (rt > rs) | ((rt == rs) & (t0 + k < s));
                }
        }
        if (s < S && rank < left) J.prefix[s + 1] += 1;
    }
    __syncthreads();
    const int per = (S + bs - 1) / bs;
    const int a = min(S, tid * per), b = min(S, a + per);
    unsigned long long local = 0;
    for (int k = a; k < b; ++k) local += J.prefix[k + 1];
    unsigned long long run = block_exclusive_u64(local, red);
    // with the prefix sums, the incident energy of the run as the transport
    // rounds it history by history (n_s units(E_s w_s)) and the history count
    unsigned long long inc = 0;
    for (int k = a; k < b; ++k) {
        const unsigned long long n = J.prefix[k + 1];
        const float w = n ? (float)((double)J.protons[k] * (double)N / ((double)n * (double)W)) : 0.0f;
        J.wh[k] = w;
        inc += n * to_units(J.spot[k].z * w);
        run += n;
        J.prefix[k + 1] = run;
    }
    inc = block_sum_u64(inc, red);
    if (tid == 0) {
        J.prefix[0] = 0;
        J.ledger[LED_W] = W;
        J.ledger[LED_INC] = inc;
        J.ledger[LED_HIST] = N;
    }
}

// ---------------------------------------------------------------- transport
namespace {

__device__ __forceinline__ float highland_g(float u)
{
    if (!(u > 0.0f)) return 0.0f;
    const float t = fmaf(kHighlandB, __logf(u), 1.0f);
    return u * t * t;
}

// Linear interpolation on the uniform energy grid for 0 <= e < kEmax: spot
// energies are at most 250 MeV (checked where plans enter) and a history's
// energy only decreases, so the index needs no clamp.  The two values of an
// entry are interpolated by one paired FMA.
__device__ __forceinline__ float2 lerp_e_in(const float4 *t, float e)
{
    const float x = e * kInvDE;
    const int i = (int)x;
    const float f = x - (float)i;
    const float4 a = t[i];
    return __ffma2_rn(make_float2(f, f), make_float2(a.z, a.w), make_float2(a.x, a.y));
}

// Energy at a residual water range 0 <= r < kRmax (below the range of
// 250 MeV), linear on the sqrt(range) grid.
__device__ __forceinline__ float energy_at_range_in(const float2 *er, float r, float inv_ds)
{
    const float x = fast_sqrt(r) * inv_ds;
    const int i = (int)x;
    const float f = x - (float)i;
    const float2 a = er[i];
    return fmaf(f, a.y, a.x);
}

// Box-Muller pair of box_muller(), its two products as one paired multiply.
__device__ __forceinline__ float2 box_muller2(float ua, float ub)
{
    const float t = fmaxf(-2.0f * __logf(ua), 1e-30f);
    const float r = t * rsqrtf(t);
    const float a = __fmaf_rn(6.28318530717958647f, ub, -3.14159265358979324f);
    float s, c;
    __sincosf(a, &s, &c);
    return __fmul2_rn(make_float2(-r, -r), make_float2(c, s));
}

}  // namespace

// Persistent kernel: every warp pulls `chunk` consecutive work items (one
// history each) from a global counter and keeps its 32 lanes busy.  Births
// are made 32 at a time by the whole warp (every lane computes the birth of
// one work item; those that start inside the grid go, ranked by ballot, into
// the warp's buffer in shared memory), and a lane whose history ends takes
// the next buffered birth at once.  A birth therefore runs with all lanes
// active, and a dead lane idles only while its warp finishes the step.  The
// loop ends when the counter passes `total`, the buffer is empty and every
// lane of the warp is idle.  Every history is a pure function of (seed,
// history index, stream), so results do not depend on the launch shape, on
// the chunking, on the buffering or on the batching.
//
// kMode kTable: the jobs come from the table `jobs` (staged in shared
// memory when `stage`), P is unused.  kSingle: one job, whose descriptor P
// is a kernel parameter (constant memory, read as instruction operands; no
// job search at birth); its counters are added in shared memory.  kShared:
// a table of jobs that agree on every per-step field before `hu` (grid
// size, voxel size, SPR scale, physics, step limit, Philox round keys),
// which come from P; each step reads only its job's grid, tally and stream
// from the table.
//
// kPhys >= 0 fixes the physics mask at compile time (the job's mask must
// equal it) and kMat fixes the material source (1: every job has a (rho,
// SPR) grid; 2: every job reads HU + table); -1 reads them from the job.
// A fixed value drops the per-step branches on it; the arithmetic, and so
// every result, is the same.
// kGeom: a table of jobs that agree on the grid, physics and step limit
// (views of one grid under different seeds or SPR scales: trials, serving
// steps), which come from P; the round keys and SPR scale come from the
// job's entry with its grid, tally and stream.
enum { kTable = 0, kSingle = 1, kShared = 2, kGeom = 3 };
static_assert(kTable == kLaunchTable && kSingle == kLaunchSingle && kShared == kLaunchShared &&
              kGeom == kLaunchGeom, "launch modes");
template <int kMode, int kPhys, int kMat>
__device__ __forceinline__ void transport_body(const TJob *__restrict__ jobs, const TJob &P, int n_jobs,
                                               unsigned long long total,
                                               unsigned long long *__restrict__ counter,
                                               const Tables *__restrict__ gtab, float inv_ds,
                                               unsigned chunk, int stage)
{
    extern __shared__ int4 smem[];
    const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5;
    const size_t birth_bytes = birth_smem(blockDim.x);
    float *bbuf = reinterpret_cast<float *>(reinterpret_cast<char *>(smem) + kSmemTables);
    TJob *s_jobs = reinterpret_cast<TJob *>(reinterpret_cast<char *>(smem) + kSmemTables + birth_bytes);
    const bool table_staged = kMode != kSingle && stage != 0;  // transport_smem(n_jobs) + birth_smem(block)
    const bool staged = kMode == kSingle || table_staged;     // per-job counters in shared memory
    unsigned long long *s_led = reinterpret_cast<unsigned long long *>(
        reinterpret_cast<char *>(smem) + kSmemTables + birth_bytes + (table_staged ? n_jobs : 0) * sizeof(TJob));
    const int n_led = kMode == kSingle ? 1 : n_jobs;
    {
        const int4 *src = reinterpret_cast<const int4 *>(gtab);
        for (int i = threadIdx.x; i < (int)(kSmemTables / 16); i += blockDim.x) smem[i] = src[i];
        if (table_staged) {
            const int words = n_jobs * (int)(sizeof(TJob) / 4);
            const int *js = reinterpret_cast<const int *>(jobs);
            int *jd = reinterpret_cast<int *>(s_jobs);
            for (int i = threadIdx.x; i < words; i += blockDim.x) jd[i] = js[i];
        }
        if (staged)
            for (int i = threadIdx.x; i < n_led * 4; i += blockDim.x) s_led[i] = 0ull;
    }
    __syncthreads();
    // re, hs, er from shared memory; mat (beyond the staged part) from global
    const Tables &T = *reinterpret_cast<const Tables *>(smem);
    const float2 *__restrict__ mat = gtab->mat;
    // job descriptors: the parameter, shared memory when staged, else global
    const TJob *jt = table_staged ? s_jobs : jobs;
    // job_of: the per-step fields shared by the launch's jobs (and everything
    // a birth reads); own_of: the job's grid, tally, stream and ledger
    auto job_of = [&](int j) -> const TJob & { return kMode == kTable ? jt[j] : P; };
    // the per-step fields that kGeom takes from the job: round keys, SPR scale
    auto key_of = [&](int j) -> const TJob & { return kMode == kTable || kMode == kGeom ? jt[j] : P; };
    auto own_of = [&](int j) -> const TJob & { return kMode == kSingle ? P : jt[j]; };
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    // this warp's birth buffer: word f of slot k is wb[f * plane + k] (one
    // plane of 32 slots per word and warp, so lanes writing consecutive
    // slots hit distinct banks)
    float *wb = bbuf + warp * 32;
    const int plane = nwarps * 32;

    // Per-job counters: escaped and removed energy, steps, flags.  Staged
    // launches add them in shared memory and flush once per block.
    auto led_add = [&](int j, int which, unsigned long long v) {
        if (!v) return;
        if (staged) atomicAdd(s_led + 4 * j + which, v);
        else atomicAdd(jobs[j].ledger + (which == 0 ? LED_ESC : which == 1 ? LED_REM : LED_STEPS), v);
    };

    // per-lane history state; wq is the history weight times the tally
    // quantum 2^24 (an exact scaling), so a deposit e is e * wq units
    bool alive = false;
    float px = 0, py = 0, pz = 0, ux = 0, uy = 0, uz = 0, E = 0, eta = 0, uth = 0, gth = 0, wq = 0;
    int ix = 0, iy = 0, iz = 0;
    unsigned step = 0;
    unsigned long long h = 0;
    int job = 0;

    // warp-uniform queue state
    unsigned long long pool_next = 0, pool_end = 0;
    bool queue_done = false;
    int n_buf = 0;                                   // births waiting in this warp's buffer

    for (;;) {
        // ---------------- idle lanes take the next born histories; when the
        // buffer is empty the whole warp births the next 32 work items
        unsigned dead = __ballot_sync(kFull, !alive);
        while (dead) {
            if (n_buf == 0) {
                if (queue_done) break;
                if (pool_next >= pool_end) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(counter, (unsigned long long)chunk);
                    base = __shfl_sync(kFull, base, 0);
                    if (base >= total) { queue_done = true; break; }
                    pool_next = base;
                    pool_end = min(base + (unsigned long long)chunk, total);
                }
                const unsigned long long avail = pool_end - pool_next;
                bool ok = false;
                float bpx = 0, bpy = 0, bpz = 0, bux = 0, buy = 0, buz = 0, bE = 0, beta = 0, bwq = 0;
                int bix = 0, biy = 0, biz = 0, bjob = 0;
                unsigned long long bh = 0;
                if (lane < avail) {
                    const unsigned long long w = pool_next + lane;
                    int lo = 0;
                    if (kMode != kSingle) {
                        int hi = n_jobs;
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (jt[mid].work_begin <= w) lo = mid; else hi = mid;
                        }
                    }
                    const TJob &J = own_of(lo);
                    bjob = lo;
                    bh = J.hist_begin + spread_history(w - J.work_begin, J.n_work, J.spread_log2);
                    const int S = J.n_spots;
                    const unsigned long long *prefix = J.prefix;
                    if (bh < prefix[S]) {
                        int a = 0, b = S;
                        while (b - a > 1) {
                            const int m = (a + b) >> 1;
                            if (prefix[m] <= bh) a = m; else b = m;
                        }
                        const float4 sp = J.spot[a];
                        bwq = J.wh[a] * kQuantum;
                        bE = sp.z;
                        const U6 u = uniforms6(philox4x32_10(
                            make_uint4(0u, (unsigned)bh, (unsigned)(bh >> 32), J.stream), J.key0, J.key1));
                        const float2 z = box_muller(u.u[0], u.u[1]);
                        beta = -__logf(u.u[2]);
                        // the spot's field may enter along its own grid axis
                        int ax = J.beam_axis, sg = J.beam_sign;
                        if (J.spot_dir) {
                            const unsigned code = J.spot_dir[a];
                            ax = (int)(code >> 1);
                            sg = (code & 1u) ? 1 : -1;
                        }
                        const float lb = sp.x - J.o[ax == 0 ? 1 : 0] + sp.w * z.x;
                        const float lc = sp.y - J.o[ax == 2 ? 1 : 2] + sp.w * z.y;
                        const int nx = J.nx, ny = J.ny, nz = J.nz;
                        const float dx = J.dx, dy = J.dy, dz = J.dz;
                        bool inside;
                        if (ax == 2) {
                            inside = lb >= 0.0f && lb < nx * dx && lc >= 0.0f && lc < ny * dy;
                            bpx = lb; bpy = lc; bpz = sg > 0 ? 0.0f : nz * dz; buz = (float)sg;
                            bix = (int)floorf(bpx * J.idx); biy = (int)floorf(bpy * J.idy); biz = sg > 0 ? 0 : nz - 1;
                        } else if (ax == 1) {
                            inside = lb >= 0.0f && lb < nx * dx && lc >= 0.0f && lc < nz * dz;
                            bpx = lb; bpz = lc; bpy = sg > 0 ? 0.0f : ny * dy; buy = (float)sg;
                            bix = (int)floorf(bpx * J.idx); biz = (int)floorf(bpz * J.idz); biy = sg > 0 ? 0 : ny - 1;
                        } else {
                            inside = lb >= 0.0f && lb < ny * dy && lc >= 0.0f && lc < nz * dz;
                            bpy = lb; bpz = lc; bpx = sg > 0 ? 0.0f : nx * dx; bux = (float)sg;
                            biy = (int)floorf(bpy * J.idy); biz = (int)floorf(bpz * J.idz); bix = sg > 0 ? 0 : nx - 1;
                        }
                        // guard the floor against rounding at the far faces
                        bix = min(max(bix, 0), nx - 1); biy = min(max(biy, 0), ny - 1); biz = min(max(biz, 0), nz - 1);
                        if (inside) ok = true;
                        else led_add(bjob, 0, __float2ull_rn(bE * bwq));
                    }
                }
                pool_next += min(32ull, avail);
                const unsigned okm = __ballot_sync(kFull, ok);
                if (ok) {
                    float *e = wb + __popc(okm & lt_mask);
                    e[0 * plane] = bpx; e[1 * plane] = bpy; e[2 * plane] = bpz;
                    e[3 * plane] = bux; e[4 * plane] = buy; e[5 * plane] = buz;
                    e[6 * plane] = bE; e[7 * plane] = beta; e[8 * plane] = bwq;
                    e[9 * plane] = __int_as_float(bix); e[10 * plane] = __int_as_float(biy);
                    e[11 * plane] = __int_as_float(biz); e[12 * plane] = __int_as_float(bjob);
                    e[13 * plane] = __uint_as_float((unsigned)bh); e[14 * plane] = __uint_as_float((unsigned)(bh >> 32));
                }
                n_buf = __popc(okm);
                __syncwarp();
                continue;
            }
            const int take = min(__popc(dead), n_buf);
            const int rank = __popc(dead & lt_mask);
            if (!alive && rank < take) {
                const float *e = wb + (n_buf - 1 - rank);
                px = e[0 * plane]; py = e[1 * plane]; pz = e[2 * plane];
                ux = e[3 * plane]; uy = e[4 * plane]; uz = e[5 * plane];
                E = e[6 * plane]; eta = e[7 * plane]; wq = e[8 * plane];
                ix = __float_as_int(e[9 * plane]); iy = __float_as_int(e[10 * plane]);
                iz = __float_as_int(e[11 * plane]);
                if (kMode != kSingle) job = __float_as_int(e[12 * plane]);
                h = (unsigned long long)__float_as_uint(e[13 * plane]) |
                    ((unsigned long long)__float_as_uint(e[14 * plane]) << 32);
                uth = 0.0f; gth = 0.0f; step = 0;
                alive = true;
            }
            n_buf -= take;
            __syncwarp();
            dead = __ballot_sync(kFull, !alive);
        }
        if (dead == kFull) break;                    // the queue and the buffer are empty
        if (!alive) continue;

        // ---------------- one condensed-history step
        const TJob &J = job_of(job);
        const TJob &Jo = own_of(job);
        const int nx = J.nx, ny = J.ny;
        const int vox = (iz * ny + iy) * nx + ix;
        float2 m;
        // the grid is read at random voxels (few L1 hits): through L2 only,
        // so L1 keeps the job descriptors and the HU table
        if (kMat == 1 || (kMat < 0 && Jo.matg)) {
            m = __ldcg(Jo.matg + vox);
        } else {
            const int hv = min(max((int)__ldcg(Jo.hu + vox), kHuMin), kHuMax);
            m = __ldg(mat + (hv - kHuMin));
        }
        const float rho = m.x;
        const TJob &Jk = key_of(job);
        const float spr = m.y * Jk.spr_scale;
        const float inv_spr = __fdividef(1.0f, spr);
        const float2 re0 = lerp_e_in(T.re, E);
        const float R0 = re0.x;
        ++step;
        // this step's random numbers: independent of the geometry below, so
        // the generator's rounds can interleave with the table lookups
        const U6 u = uniforms6(philox_rk(
            make_uint4(step, (unsigned)h, (unsigned)(h >> 32), Jo.stream), Jk.rk));
        const float q = R0 * inv_spr;                  // residual range in the medium
        if (q <= kSmin) {                              // residual range below s_min
            atomicAdd(Jo.tally + vox, __float2ull_rn(E * wq));
            led_add(job, 2, step);
            alive = false;
            continue;
        }
        const float dx = J.dx, dy = J.dy, dz = J.dz;
        // distance to the faces of the current voxel (ties: lowest axis):
        // (face - p) / u towards the face the direction points at, none
        // along an axis the direction does not move on
        const float inf = __int_as_float(0x7f800000);
        const float bx = (float)(ux > 0.0f ? ix + 1 : ix), by = (float)(uy > 0.0f ? iy + 1 : iy);
        const float bz = (float)(uz > 0.0f ? iz + 1 : iz);
        const float2 dxy = __fmul2_rn(__ffma2_rn(make_float2(bx, by), make_float2(dx, dy), make_float2(-px, -py)),
                                      make_float2(__fdividef(1.0f, ux), __fdividef(1.0f, uy)));
        float tx = ux != 0.0f ? dxy.x : inf;
        float ty = uy != 0.0f ? dxy.y : inf;
        float tz = uz != 0.0f ? __fmaf_rn(bz, dz, -pz) * __fdividef(1.0f, uz) : inf;
        tx = fmaxf(tx, 0.0f); ty = fmaxf(ty, 0.0f); tz = fmaxf(tz, 0.0f);
        int across = 0;
        float dbound = tx;
        if (ty < dbound) { dbound = ty; across = 1; }
        if (tz < dbound) { dbound = tz; across = 2; }
        // the step ends at the voxel boundary or after the physics length
        // (kFstep R0 / SPR: the factor 1/4 scales exactly)
        float s = fmaxf(kFstep * q, kSmin);
        bool geom = false;
        if (dbound <= s) { s = dbound; geom = true; }

        float sw = s * spr;                              // water-equivalent mm
        float E1c = energy_at_range_in(T.er, R0 - sw, inv_ds);
        float Emean = 0.5f * (E + E1c);
        float2 hs = lerp_e_in(T.hs, Emean);
        const unsigned physics = kPhys >= 0 ? (unsigned)kPhys : J.physics;
        bool nuclear = false;
        if (physics & 4u) {
            const float tau = hs.y * sw;
            if (hs.y > 0.0f && tau >= eta) {
                nuclear = true;
                sw = __fdividef(eta, hs.y);
                s = sw * inv_spr;
                geom = false;
                E1c = energy_at_range_in(T.er, R0 - sw, inv_ds);
            } else {
                eta -= tau;
            }
        }
        float dE = E - E1c;
        if (physics & 1u) {
            // Bohr straggling: a lognormal loss with the CSDA loss as its
            // mean and the Bohr variance, for any step length
            const float zA = box_muller_first(u.u[0], u.u[1]);
            dE = fminf(straggle_loss(dE, re0.y * sw, zA), E);
        }
        const float E1 = E - dE;
        dE = E - E1;

        if (nuclear || E1 <= kEcut) {
            float local = E;                              // stop: dE + E1
            if (nuclear) {
                local = dE + kFloc * E1;
                led_add(job, 1, __float2ull_rn((E1 - kFloc * E1) * wq));
            }
            atomicAdd(Jo.tally + vox, __float2ull_rn(local * wq));
            led_add(job, 2, step);
            alive = false;
            continue;
        }
        atomicAdd(Jo.tally + vox, __float2ull_rn(dE * wq));

        // multiple Coulomb scattering over the step (cumulative Highland);
        // the two transverse planes as float2 pairs (y1, y2) and (t1, t2)
        float2 y = make_float2(0.0f, 0.0f), t = make_float2(0.0f, 0.0f);
        if (physics & 2u) {
            const float u1 = fmaf(s * rho, kInvX0, uth);
            const float g1 = highland_g(u1);
            const float th2 = highland_coeff(hs.x) * (g1 - gth);
            uth = u1; gth = g1;
            const float th0 = fast_sqrt(th2);
            const float2 zu = box_muller2(u.u[2], u.u[3]);
            const float2 zv = box_muller2(u.u[4], u.u[5]);
            const float st = s * th0;
            // y = s th0 (z1 / sqrt(12) + z2 / 2), t = th0 z2, per plane
            const float2 g = __ffma2_rn(make_float2(zu.x, zv.x), make_float2(kInvSqrt12, kInvSqrt12),
                                        __fmul2_rn(make_float2(0.5f, 0.5f), make_float2(zu.y, zv.y)));
            y = __fmul2_rn(make_float2(st, st), g);
            t = __fmul2_rn(make_float2(th0, th0), make_float2(zu.y, zv.y));
        }
        // transverse frame (Duff et al., JCGT 2017)
        const float sgn = uz >= 0.0f ? 1.0f : -1.0f;
        const float fa = __fdividef(-1.0f, sgn + uz);
        const float fb = ux * uy * fa;
        const float e1x = fmaf(sgn * ux * ux, fa, 1.0f), e1y = sgn * fb, e1z = -sgn * ux;
        const float e2x = fb, e2y = fmaf(uy * uy, fa, sgn), e2z = -uy;
        const float ux0 = ux, uy0 = uy, uz0 = uz;
        {
            const float2 pxy = __ffma2_rn(make_float2(s, s), make_float2(ux, uy),
                                          __ffma2_rn(make_float2(y.x, y.x), make_float2(e1x, e1y),
                                                     __ffma2_rn(make_float2(y.y, y.y), make_float2(e2x, e2y),
                                                                make_float2(px, py))));
            pz = fmaf(s, uz, fmaf(y.x, e1z, fmaf(y.y, e2z, pz)));
            const float2 uxy = __ffma2_rn(make_float2(t.x, t.x), make_float2(e1x, e1y),
                                          __ffma2_rn(make_float2(t.y, t.y), make_float2(e2x, e2y),
                                                     make_float2(ux, uy)));
            uz = fmaf(t.x, e1z, fmaf(t.y, e2z, uz));
            px = pxy.x; py = pxy.y; ux = uxy.x; uy = uxy.y;
        }
        const float nrm = rsqrtf(ux * ux + uy * uy + uz * uz);
        {
            const float2 uxy = __fmul2_rn(make_float2(ux, uy), make_float2(nrm, nrm));
            ux = uxy.x; uy = uxy.y;
            uz *= nrm;
        }
        E = E1;

        // voxel update: the crossed axis steps by one and its coordinate is
        // put on the crossed face; every other axis keeps its index while the
        // position stays inside the voxel's closed extent and takes
        // floor(p / d) once the lateral displacement carried it outside
        if (geom && across == 0) {
            if (ux0 > 0.0f) { ix += 1; px = ix * dx; } else { px = ix * dx; ix -= 1; }
        } else {
            const float2 ext = __fmul2_rn(make_float2((float)ix, (float)(ix + 1)), make_float2(dx, dx));
            if (!(px >= ext.x && px <= ext.y)) ix = (int)floorf(px * J.idx);
        }
        if (geom && across == 1) {
            if (uy0 > 0.0f) { iy += 1; py = iy * dy; } else { py = iy * dy; iy -= 1; }
        } else {
            const float2 ext = __fmul2_rn(make_float2((float)iy, (float)(iy + 1)), make_float2(dy, dy));
            if (!(py >= ext.x && py <= ext.y)) iy = (int)floorf(py * J.idy);
        }
        if (geom && across == 2) {
            if (uz0 > 0.0f) { iz += 1; pz = iz * dz; } else { pz = iz * dz; iz -= 1; }
        } else {
            const float2 ext = __fmul2_rn(make_float2((float)iz, (float)(iz + 1)), make_float2(dz, dz));
            if (!(pz >= ext.x && pz <= ext.y)) iz = (int)floorf(pz * J.idz);
        }
        // leaving the grid, or the step limit reached (checked with the exit
        // so that a step pays one rare branch): the energy escapes
        const bool outside = (unsigned)ix >= (unsigned)nx || (unsigned)iy >= (unsigned)ny ||
                             (unsigned)iz >= (unsigned)J.nz;
        if (outside || step >= J.max_steps) {
            led_add(job, 0, __float2ull_rn(E * wq));
            led_add(job, 2, step);
            if (!outside) {
                if (staged) atomicOr(s_led + 4 * job + 3, (unsigned long long)FLAG_STEPLIMIT);
                else atomicOr(jobs[job].ledger + LED_FLAGS, (unsigned long long)FLAG_STEPLIMIT);
            }
            alive = false;
        }
    }
    if (staged) {
        __syncthreads();
        for (int i = threadIdx.x; i < n_led * 4; i += blockDim.x) {
            const unsigned long long v = s_led[i];
            if (!v) continue;
            const int j = i >> 2, which = i & 3;
            unsigned long long *led = own_of(j).ledger;
            if (which == 3) atomicOr(led + LED_FLAGS, v);
            else atomicAdd(led + (which == 0 ? LED_ESC : which == 1 ? LED_REM : LED_STEPS), v);
        }
    }
}

// Two register budgets of the same kernel: up to 128 registers per thread
// (blocks of at most 512 threads) or 64 (blocks up to 1024 threads, more
// resident warps).  The autotuner picks; results are equal.  k_transport1*
// run one job given as a parameter; k_transportS* a table of jobs whose
// per-step fields come from the parameter `common`; k_transport* a table.
// Each comes in the specialisations of transport_spec().
template <int P, int M>
__global__ void __launch_bounds__(512, 1)
k_transport(const TJob *__restrict__ jobs, int n_jobs, unsigned long long total,
            unsigned long long *__restrict__ counter, const Tables *__restrict__ gtab, float inv_ds,
            unsigned chunk, int stage)
{
    transport_body<kTable, P, M>(jobs, *jobs, n_jobs, total, counter, gtab, inv_ds, chunk, stage);
}

template <int P, int M>
__global__ void __launch_bounds__(1024, 1)
k_transport_r64(const TJob *__restrict__ jobs, int n_jobs, unsigned long long total,
                unsigned long long *__restrict__ counter, const Tables *__restrict__ gtab,
                float inv_ds, unsigned chunk, int stage)
{
    transport_body<kTable, P, M>(jobs, *jobs, n_jobs, total, counter, gtab, inv_ds, chunk, stage);
}

template <int P, int M>
__global__ void __launch_bounds__(512, 1)
k_transport1(const __grid_constant__ TJob job, unsigned long long total, unsigned long long *__restrict__ counter,
             const Tables *__restrict__ gtab, float inv_ds, unsigned chunk)
{
    transport_body<kSingle, P, M>(nullptr, job, 1, total, counter, gtab, inv_ds, chunk, 0);
}

template <int P, int M>
__global__ void __launch_bounds__(1024, 1)
k_transport1_r64(const __grid_constant__ TJob job, unsigned long long total,
                 unsigned long long *__restrict__ counter, const Tables *__restrict__ gtab, float inv_ds,
                 unsigned chunk)
{
    transport_body<kSingle, P, M>(nullptr, job, 1, total, counter, gtab, inv_ds, chunk, 0);
}

template <int P, int M>
__global__ void __launch_bounds__(512, 1)
k_transportS(const __grid_constant__ TJob common, const TJob *__restrict__ jobs, int n_jobs, unsigned long long total,
             unsigned long long *__restrict__ counter, const Tables *__restrict__ gtab, float inv_ds,
             unsigned chunk, int stage)
{
    transport_body<kShared, P, M>(jobs, common, n_jobs, total, counter, gtab, inv_ds, chunk, stage);
}

template <int P, int M>
__global__ void __launch_bounds__(1024, 1)
k_transportS_r64(const __grid_constant__ TJob common, const TJob *__restrict__ jobs, int n_jobs,
                 unsigned long long total, unsigned long long *__restrict__ counter,
                 const Tables *__restrict__ gtab, float inv_ds, unsigned chunk, int stage)
{
    transport_body<kShared, P, M>(jobs, common, n_jobs, total, counter, gtab, inv_ds, chunk, stage);
}

template <int P, int M>
__global__ void __launch_bounds__(512, 1)
k_transportG(const __grid_constant__ TJob common, const TJob *__restrict__ jobs, int n_jobs, unsigned long long total,
             unsigned long long *__restrict__ counter, const Tables *__restrict__ gtab, float inv_ds,
             unsigned chunk, int stage)
{
    transport_body<kGeom, P, M>(jobs, common, n_jobs, total, counter, gtab, inv_ds, chunk, stage);
}

template <int P, int M>
__global__ void __launch_bounds__(1024, 1)
k_transportG_r64(const __grid_constant__ TJob common, const TJob *__restrict__ jobs, int n_jobs,
                 unsigned long long total, unsigned long long *__restrict__ counter,
                 const Tables *__restrict__ gtab, float inv_ds, unsigned chunk, int stage)
{
    transport_body<kGeom, P, M>(jobs, common, n_jobs, total, counter, gtab, inv_ds, chunk, stage);
}

namespace {
// (kPhys, kMat) of each specialisation
template <int S> struct SpecArgs;
template <> struct SpecArgs<kSpecGeneric> { static constexpr int P = -1, M = -1; };
template <> struct SpecArgs<kSpecFullGrid> { static constexpr int P = 7, M = 1; };
template <> struct SpecArgs<kSpecFullHu> { static constexpr int P = 7, M = 2; };

template <int S>
const void *kernel_of(int mode, int regs)
{
    constexpr int P = SpecArgs<S>::P, M = SpecArgs<S>::M;
    if (mode == kSingle) return regs ? (const void *)k_transport1_r64<P, M> : (const void *)k_transport1<P, M>;
    if (mode == kShared) return regs ? (const void *)k_transportS_r64<P, M> : (const void *)k_transportS<P, M>;
    if (mode == kGeom) return regs ? (const void *)k_transportG_r64<P, M> : (const void *)k_transportG<P, M>;
    return regs ? (const void *)k_transport_r64<P, M> : (const void *)k_transport<P, M>;
}

template <int S>
void launch_spec(const TransportLaunch &L)
{
    constexpr int P = SpecArgs<S>::P, M = SpecArgs<S>::M;
    const dim3 g(L.grid), b(L.block);
    if (L.mode == kSingle && L.regs)
        k_transport1_r64<P, M><<<g, b, L.smem, L.stream>>>(*L.job0, L.total, L.counter, L.tab, L.inv_ds, L.chunk);
    else if (L.mode == kSingle)
        k_transport1<P, M><<<g, b, L.smem, L.stream>>>(*L.job0, L.total, L.counter, L.tab, L.inv_ds, L.chunk);
    else if (L.mode == kShared && L.regs)
        k_transportS_r64<P, M><<<g, b, L.smem, L.stream>>>(*L.job0, L.d_jobs, L.n_jobs, L.total, L.counter, L.tab,
                                                            L.inv_ds, L.chunk, L.stage);
    else if (L.mode == kShared)
        k_transportS<P, M><<<g, b, L.smem, L.stream>>>(*L.job0, L.d_jobs, L.n_jobs, L.total, L.counter, L.tab,
                                                        L.inv_ds, L.chunk, L.stage);
    else if (L.mode == kGeom && L.regs)
        k_transportG_r64<P, M><<<g, b, L.smem, L.stream>>>(*L.job0, L.d_jobs, L.n_jobs, L.total, L.counter, L.tab,
                                                            L.inv_ds, L.chunk, L.stage);
    else if (L.mode == kGeom)
        k_transportG<P, M><<<g, b, L.smem, L.stream>>>(*L.job0, L.d_jobs, L.n_jobs, L.total, L.counter, L.tab,
                                                        L.inv_ds, L.chunk, L.stage);
    else if (L.regs)
        k_transport_r64<P, M><<<g, b, L.smem, L.stream>>>(L.d_jobs, L.n_jobs, L.total, L.counter, L.tab, L.inv_ds,
                                                           L.chunk, L.stage);
    else
        k_transport<P, M><<<g, b, L.smem, L.stream>>>(L.d_jobs, L.n_jobs, L.total, L.counter, L.tab, L.inv_ds,
                                                       L.chunk, L.stage);
}
}  // namespace

int transport_spec(const TJob *jobs, int n)
{
    bool full = n > 0, grid = true, hu = true;
    for (int j = 0; j < n; ++j) {
        full = full && jobs[j].physics == 7u;
        grid = grid && jobs[j].matg != nullptr;
        hu = hu && jobs[j].matg == nullptr;
    }
    if (!full) return kSpecGeneric;
    return grid ? kSpecFullGrid : hu ? kSpecFullHu : kSpecGeneric;
}

const void *transport_kernel(int mode, int regs, int spec)
{
    if (spec == kSpecFullGrid) return kernel_of<kSpecFullGrid>(mode, regs);
    if (spec == kSpecFullHu) return kernel_of<kSpecFullHu>(mode, regs);
    return kernel_of<kSpecGeneric>(mode, regs);
}

cudaError_t transport_launch(const TransportLaunch &L)
{
    if (L.spec == kSpecFullGrid) launch_spec<kSpecFullGrid>(L);
    else if (L.spec == kSpecFullHu) launch_spec<kSpecFullHu>(L);
    else launch_spec<kSpecGeneric>(L);
    return cudaGetLastError();
}

cudaError_t transport_allow_smem()
{
    // the attribute is a per-device property of each kernel: set it once per
    // device (24 calls), not on every launch
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    const int bytes = (int)(kSmemTransportMax + birth_smem(1024));
    for (int spec = 0; spec < 3; ++spec)
        for (int mode = 0; mode < 4; ++mode)
            for (int regs = 0; regs < 2; ++regs) {
                e = cudaFuncSetAttribute(transport_kernel(mode, regs, spec),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
                if (e != cudaSuccess) return e;
            }
    done.fetch_or(bit, std::memory_order_release);
    return cudaSuccess;
}

// ------------------------------------------------------------- self-tests
__global__ void k_debug_philox(const uint4 *ctr, const uint2 *key, uint4 *out, float *uni, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 w = philox4x32_10(ctr[i], key[i].x, key[i].y);
    out[i] = w;
    const U6 u = uniforms6(w);
    for (int k = 0; k < 6; ++k) uni[6 * i + k] = u.u[k];
}

__global__ void k_debug_tables(const Tables *tab, float inv_ds, const float *e, int n, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 re = lerp_e(tab->re, e[i]);
    const float2 hs = lerp_e(tab->hs, e[i]);
    out[5 * i + 0] = re.x;
    out[5 * i + 1] = energy_at_range(tab->er, re.x, inv_ds);
    out[5 * i + 2] = re.y;
    out[5 * i + 3] = highland_coeff(hs.x);
    out[5 * i + 4] = hs.y;
}

// -------------------------------------------------------------- normalise
// D_i = tally_i 2^-24 MeV x (W/N) x 1.602176634e-13 J/MeV / (rho_i V 1e-3 kg)
__global__ void k_normalise(const NormJob *__restrict__ jobs)
{
    const NormJob J = jobs[blockIdx.y];
    const unsigned long long W = J.ledger[LED_W];
    const double factor = (W == 0 || J.n_hist == 0) ? 0.0
        : (double)W / (double)J.n_hist * 1.602176634e-10 / (16777216.0 * J.voxel_cm3);
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned long long dep = 0;
    // four voxels per pass, their tallies loaded together
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < J.nvox; i0 += 4 * stride) {
        unsigned long long t[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long i = i0 + k * stride;
            t[k] = i < J.nvox ? J.tally[i] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long i = i0 + k * stride;
            if (i >= J.nvox) break;
            dep += t[k];
            // most voxels of a beam's grid hold no energy: their dose is +0
            // without the FP64 quotient (or the density read)
            J.dose[i] = t[k] ? (float)div64((double)t[k] * factor, (double)J.rho[i]) : 0.0f;
        }
    }
    dep = warp_sum_u64(dep);
    if ((threadIdx.x & 31) == 0 && dep) atomicAdd(J.ledger + LED_DEP, dep);
}

}  // namespace dose
