// Energy/mass-transfer accumulation (Sec. 2.D.2, Eqs. 4-6 of Pepin et al.)
// and the phase sum of Eq. 2.
//
//   k_reach     per source phase: the largest rho_j D_j (fixed-point
//               scale), the box of the voxels that carry dose and the largest
//               displacement per axis (also run before the DIM)
//   k_dvf4      one source phase's field, x/y/z planes -> one float4 per
//               voxel, over the nodes its reach reads
//   k_emtm      a thread per source voxel j within reach of dose: split j into
//               nsx x nsy x nsz subvoxels, move each centre by the phase's DVF
//               (trilinear between voxel centres, edge-clamped; one 16-byte
//               load per node) and add the subvoxel's mass rho_j and energy
//               rho_j D_j (both in units of the common subvoxel volume) to the
//               reference voxel whose half-open cell holds it.  Consecutive
//               subvoxels landing in the same voxel are summed in registers
//               and pushed with one pair of 64-bit integer atomics, so the
//               sums are exact and order-free.
//   k_emtm_zero E and M cleared where the sum reads them
//   k_emtm_sum  D_i = D_i^R + sum_S E_i^S / M_i^S (0 where M = 0), masked.
//
// Source voxels out of reach (reach_box with mult 2) are not pushed: every
// voxel they can reach receives no energy, so E_i^S = 0 and the term adds
// exactly zero whatever M_i^S holds.  The result is the same as pushing
// every voxel; only the counters of pushed and dropped subvoxels count
// the voxels within reach.
//
// The target voxel is decided in single precision with the rounding order
// written out below (no contraction; the displacement goes to voxel units
// through the FP32 reciprocal of the voxel size), so it is reproducible bit
// for bit.
#include <cuda_runtime.h>
#include <climits>
#include <cmath>
#include "engine.cuh"
#include "kernels.h"

namespace dose {

namespace {
constexpr int kMassShift = 40;   // mass units: rho x 2^40
constexpr int kEnergyBits = 40;  // energy units: rho D scaled so max(rho D) < 2^40

__device__ __forceinline__ int energy_shift(unsigned maxbits)
{
    if (maxbits == 0) return 0;
    int e;
    frexpf(__uint_as_float(maxbits), &e);          // max < 2^e
    return kEnergyBits - e;
}

__device__ __forceinline__ float lerp_rn(float a, float b, float t)
{
    return __fadd_rn(a, __fmul_rn(t, __fsub_rn(b, a)));
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
}  // namespace

// A warp per row (y, z) of the grid, its lanes along x (coalesced).
__global__ void k_reach(ReachArgs a)
{
    const int p = blockIdx.y;
    if (p == a.ref) return;
    const size_t nvox = (size_t)a.nx * a.ny * a.nz;
    const float *d = a.dose + (size_t)p * nvox;
    const float *r = a.rho ? a.rho + (size_t)p * nvox : nullptr;
    const float *u = a.dvf ? a.dvf + (size_t)p * 3 * nvox : nullptr;
    const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
    const unsigned rows = (unsigned)a.ny * (unsigned)a.nz;
    unsigned lo[3] = {UINT_MAX, UINT_MAX, UINT_MAX}, hi[3] = {0u, 0u, 0u};   // hi: index + 1
    unsigned um[3] = {0u, 0u, 0u}, mb = 0u;
    for (unsigned row = blockIdx.x * warps + (threadIdx.x >> 5); row < rows; row += gridDim.x * warps) {
        const size_t base = (size_t)row * a.nx;
        bool hit = false;
        for (int x = lane; x < a.nx; x += 32) {
            const float dv = d[base + x];
            bool carries;
            if (r) {
                const float rv = r[base + x];
                mb = max(mb, __float_as_uint(fmaxf(rv * dv, 0.0f)));   // non-negative: bits order as values
                carries = rv > 0.0f && dv > 0.0f;
            } else {
                carries = dv != 0.0f;
            }
            if (carries) {
                lo[0] = min(lo[0], (unsigned)x);
                hi[0] = max(hi[0], (unsigned)x + 1u);
                hit = true;
            }
            if (u) {
                um[0] = max(um[0], __float_as_uint(fabsf(u[base + x])));
                um[1] = max(um[1], __float_as_uint(fabsf(u[nvox + base + x])));
                um[2] = max(um[2], __float_as_uint(fabsf(u[2 * nvox + base + x])));
            }
        }
        if (hit) {
            const unsigned y = row % (unsigned)a.ny, z = row / (unsigned)a.ny;
            lo[1] = min(lo[1], y); hi[1] = max(hi[1], y + 1u);
            lo[2] = min(lo[2], z); hi[2] = max(hi[2], z + 1u);
        }
    }
    unsigned *w = a.reach + (size_t)p * kReachWords;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = __reduce_min_sync(0xffffffffu, lo[k]);
        hi[k] = __reduce_max_sync(0xffffffffu, hi[k]);
        um[k] = __reduce_max_sync(0xffffffffu, um[k]);
    }
    mb = __reduce_max_sync(0xffffffffu, mb);
    if (lane == 0) {
        if (hi[0]) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                atomicMax(w + k, ~lo[k]);
                atomicMax(w + 3 + k, hi[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (um[k]) atomicMax(w + 6 + k, um[k]);
        if (a.maxbits && mb) atomicMax(a.maxbits + p, mb);
    }
}

// A grid-stride loop over the source voxels within reach (x fastest).
__global__ void k_emtm(EmtmArgs a)
{
    const int S = a.dvf4 ? a.phase : (int)blockIdx.y;
    if (S == a.ref) return;
    const VoxBox b = reach_box(a.reach + (size_t)S * kReachWords, 2, a.nx, a.ny, a.nz, a.idx, a.idy, a.idz);
    if (b.lo[0] > b.hi[0]) return;                                   // no dose in this phase
    // the subvoxel-centre fractions (k + 1/2) / n of each axis, once per block
    __shared__ float s_frac[3][64];
    for (int t = threadIdx.x; t < 3 * 64; t += blockDim.x) {
        const int ax = t >> 6, k = t & 63;
        const int n = ax == 0 ? a.nsx : ax == 1 ? a.nsy : a.nsz;
        s_frac[ax][k] = k < n ? __fdiv_rn(__fadd_rn((float)k, 0.5f), (float)n) : 0.0f;
    }
    __syncthreads();
    const long long nvox = (long long)a.nx * a.ny * a.nz;
    const unsigned bx = (unsigned)(b.hi[0] - b.lo[0] + 1), by = (unsigned)(b.hi[1] - b.lo[1] + 1);
    const unsigned nbox = bx * by * (unsigned)(b.hi[2] - b.lo[2] + 1);   // <= nvox < 2^31
    const int es = energy_shift(a.maxbits[S]);
    unsigned long long pushed = 0, dropped = 0, pairs = 0;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < nbox; k += gridDim.x * blockDim.x) {
        const unsigned row = k / bx;
        const int jx = b.lo[0] + (int)(k - row * bx);
        const int jy = b.lo[1] + (int)(row % by);
        const int jz = b.lo[2] + (int)(row / by);
        const long long j = ((long long)jz * a.ny + jy) * a.nx + jx;
        const float rho = a.rho[(size_t)S * nvox + j];
        const float dj = a.dose[(size_t)S * nvox + j];
        const double prod = fmax((double)rho * (double)dj, 0.0);
        const unsigned long long eu = __double2ull_rn(ldexp(prod, es));
        const unsigned long long mu = __double2ull_rn(ldexp((double)rho, kMassShift));
        unsigned long long *E = a.E + (size_t)S * nvox;
        unsigned long long *M = a.M + (size_t)S * nvox;
        long long cur = -1;
        unsigned long long cnt = 0;
        for (int kz = 0; kz < a.nsz; ++kz) {
            const float qz = __fsub_rn(__fadd_rn((float)jz, s_frac[2][kz]), 0.5f);
            for (int ky = 0; ky < a.nsy; ++ky) {
                const float qy = __fsub_rn(__fadd_rn((float)jy, s_frac[1][ky]), 0.5f);
                for (int kx = 0; kx < a.nsx; ++kx) {
                    const float qx = __fsub_rn(__fadd_rn((float)jx, s_frac[0][kx]), 0.5f);
                    float o[3] = {0.0f, 0.0f, 0.0f};
                    if (a.dvf4) {
                        const float fx0 = floorf(qx), fy0 = floorf(qy), fz0 = floorf(qz);
                        const float fx = __fsub_rn(qx, fx0), fy = __fsub_rn(qy, fy0), fz = __fsub_rn(qz, fz0);
                        const int kx0 = (int)fx0, ky0 = (int)fy0, kz0 = (int)fz0;
                        const int x0 = min(max(kx0, 0), a.nx - 1), x1 = min(max(kx0 + 1, 0), a.nx - 1);
                        const int y0 = min(max(ky0, 0), a.ny - 1), y1 = min(max(ky0 + 1, 0), a.ny - 1);
                        const int z0 = min(max(kz0, 0), a.nz - 1), z1 = min(max(kz0 + 1, 0), a.nz - 1);
                        const unsigned r00 = ((unsigned)z0 * a.ny + y0) * a.nx, r10 = ((unsigned)z0 * a.ny + y1) * a.nx;
                        const unsigned r01 = ((unsigned)z1 * a.ny + y0) * a.nx, r11 = ((unsigned)z1 * a.ny + y1) * a.nx;
                        const float4 n000 = __ldg(a.dvf4 + r00 + x0), n100 = __ldg(a.dvf4 + r00 + x1);
                        const float4 n010 = __ldg(a.dvf4 + r10 + x0), n110 = __ldg(a.dvf4 + r10 + x1);
                        const float4 n001 = __ldg(a.dvf4 + r01 + x0), n101 = __ldg(a.dvf4 + r01 + x1);
                        const float4 n011 = __ldg(a.dvf4 + r11 + x0), n111 = __ldg(a.dvf4 + r11 + x1);
#define EM_TRI(C) lerp_rn(lerp_rn(lerp_rn(n000.C, n100.C, fx), lerp_rn(n010.C, n110.C, fx), fy), \
                          lerp_rn(lerp_rn(n001.C, n101.C, fx), lerp_rn(n011.C, n111.C, fx), fy), fz)
                        o[0] = EM_TRI(x);
                        o[1] = EM_TRI(y);
                        o[2] = EM_TRI(z);
#undef EM_TRI
                    }
                    const float tx = __fadd_rn(__fadd_rn(qx, 0.5f), __fmul_rn(o[0], a.idx));
                    const float ty = __fadd_rn(__fadd_rn(qy, 0.5f), __fmul_rn(o[1], a.idy));
                    const float tz = __fadd_rn(__fadd_rn(qz, 0.5f), __fmul_rn(o[2], a.idz));
                    const int ix = (int)floorf(tx), iy = (int)floorf(ty), iz = (int)floorf(tz);
                    ++pushed;
                    if (ix < 0 || ix >= a.nx || iy < 0 || iy >= a.ny || iz < 0 || iz >= a.nz) {
                        ++dropped;
                        continue;
                    }
                    const long long i = ((long long)iz * a.ny + iy) * a.nx + ix;
                    if (i != cur) {
                        if (cnt) {
                            atomicAdd(E + cur, cnt * eu);
                            atomicAdd(M + cur, cnt * mu);
                            ++pairs;
                        }
                        cur = i;
                        cnt = 0;
                    }
                    ++cnt;
                }
            }
        }
        if (cnt) {
            atomicAdd(E + cur, cnt * eu);
            atomicAdd(M + cur, cnt * mu);
            ++pairs;
        }
    }
    pushed = warp_sum(pushed);
    dropped = warp_sum(dropped);
    pairs = warp_sum(pairs);
    if ((threadIdx.x & 31) == 0 && pushed) {
        atomicAdd(a.stats + 0, pushed);
        atomicAdd(a.stats + 1, dropped);
        atomicAdd(a.stats + 2, pairs);
    }
}

__global__ void k_dvf4(const float *__restrict__ src, float4 *__restrict__ dst, const unsigned *reach, int nx,
                       int ny, int nz, float idx, float idy, float idz)
{
    VoxBox b = reach_box(reach, 2, nx, ny, nz, idx, idy, idz);
    if (b.lo[0] > b.hi[0]) return;
    const int n[3] = {nx, ny, nz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {                 // the trilinear nodes of the box's subvoxels
        b.lo[ax] = max(b.lo[ax] - 1, 0);
        b.hi[ax] = min(b.hi[ax] + 1, n[ax] - 1);
    }
    const size_t nvox = (size_t)nx * ny * nz;
    const unsigned bx = (unsigned)(b.hi[0] - b.lo[0] + 1), by = (unsigned)(b.hi[1] - b.lo[1] + 1);
    const unsigned nbox = bx * by * (unsigned)(b.hi[2] - b.lo[2] + 1);
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < nbox; k += gridDim.x * blockDim.x) {
        const unsigned row = k / bx;
        const size_t i = ((size_t)(b.lo[2] + (int)(row / by)) * ny + (b.lo[1] + (int)(row % by))) * nx +
                         (b.lo[0] + (int)(k - row * bx));
        dst[i] = make_float4(src[i], src[nvox + i], src[2 * nvox + i], 0.0f);
    }
}

// Zeroes E and M of each source phase (grid.y) where mass can land: a
// pushed source voxel lies in reach_box(mult 2) and moves at most r - 1
// voxels, so every target is inside reach_box(mult 3).  Elsewhere the
// arrays are neither written nor read.
__global__ void k_emtm_zero(EmtmArgs a)
{
    const int S = blockIdx.y;
    if (S == a.ref) return;
    const VoxBox b = reach_box(a.reach + (size_t)S * kReachWords, 3, a.nx, a.ny, a.nz, a.idx, a.idy, a.idz);
    if (b.lo[0] > b.hi[0]) return;
    const size_t nvox = (size_t)a.nx * a.ny * a.nz;
    unsigned long long *E = a.E + (size_t)S * nvox, *M = a.M + (size_t)S * nvox;
    const unsigned bx = (unsigned)(b.hi[0] - b.lo[0] + 1), by = (unsigned)(b.hi[1] - b.lo[1] + 1);
    const unsigned nbox = bx * by * (unsigned)(b.hi[2] - b.lo[2] + 1);
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < nbox; k += gridDim.x * blockDim.x) {
        const unsigned row = k / bx;
        const size_t i = ((size_t)(b.lo[2] + (int)(row / by)) * a.ny + (b.lo[1] + (int)(row % by))) * a.nx +
                         (b.lo[0] + (int)(k - row * bx));
        E[i] = 0ull;
        M[i] = 0ull;
    }
}

// Dynamic shared memory: 8 ints per phase (the mult-3 reach box of each
// source phase, lo[3] and hi[3]; empty for the reference).
__global__ void k_emtm_sum(EmtmArgs a)
{
    extern __shared__ int s_box[];
    for (int S = threadIdx.x; S < a.n_phases; S += blockDim.x) {
        VoxBox b = reach_box(a.reach + (size_t)S * kReachWords, 3, a.nx, a.ny, a.nz, a.idx, a.idy, a.idz);
        if (S == a.ref) { b.lo[0] = 0; b.hi[0] = -1; }
        for (int k = 0; k < 3; ++k) {
            s_box[8 * S + k] = b.lo[k];
            s_box[8 * S + 3 + k] = b.hi[k];
        }
    }
    __syncthreads();
    const long long nvox = (long long)a.nx * a.ny * a.nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
        const unsigned iu = (unsigned)i, row = iu / (unsigned)a.nx;      // nvox < 2^31
        const int x = (int)(iu - row * (unsigned)a.nx), y = (int)(row % (unsigned)a.ny), z = (int)(row / (unsigned)a.ny);
        double acc = (double)a.dose[(size_t)a.ref * nvox + i];
        for (int S = 0; S < a.n_phases; ++S) {
            const int *bb = s_box + 8 * S;
            if (x < bb[0] || x > bb[3] || y < bb[1] || y > bb[4] || z < bb[2] || z > bb[5]) continue;
            const unsigned long long m = a.M[(size_t)S * nvox + i];
            if (m == 0) continue;
            const unsigned long long e = a.E[(size_t)S * nvox + i];
            if (e == 0) {                            // mass without energy: the quotient is +0
                acc += 0.0;
                continue;
            }
            // E / M back to Gy: times 2^(mass shift - energy shift), an exact
            // power of two built from its exponent bits
            const int k = kMassShift - energy_shift(a.maxbits[S]);
            const double q = div64((double)e, (double)m);
            acc += (k > -1000 && k < 1000) ? q * __longlong_as_double((long long)(1023 + k) << 52) : ldexp(q, k);
        }
        if (a.mask && !a.mask[i]) acc = 0.0;
        a.accum[i] = (float)acc;
    }
}

}  // namespace dose
