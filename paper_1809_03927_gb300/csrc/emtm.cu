// Energy/mass-transfer accumulation (Sec. 2.D.2, Eqs. 4-6 of Pepin et al.)
// and the phase sum of Eq. 2.
//
//   k_emtm_max  largest rho_j D_j of each source phase (fixed-point scale)
//   k_dvf4      one source phase's field, x/y/z planes -> one float4 per voxel
//   k_emtm      one thread per source voxel j of that phase: split j into
//               nsx x nsy x nsz subvoxels, move each centre by the phase's DVF
//               (trilinear between voxel centres, edge-clamped; one 16-byte
//               load per node) and add the subvoxel's mass rho_j and energy
//               rho_j D_j (both in units of the common subvoxel volume) to the
//               reference voxel whose half-open cell holds it.  Consecutive
//               subvoxels landing in the same voxel are summed in registers
//               and pushed with one pair of 64-bit integer atomics, so the
//               sums are exact and order-free.
//   k_emtm_sum  D_i = D_i^R + sum_S E_i^S / M_i^S (0 where M = 0), masked.
//
// The target voxel is decided in single precision with the rounding order
// written out below (no contraction; the displacement goes to voxel units
// through the FP32 reciprocal of the voxel size), so it is reproducible bit
// for bit.
#include <cuda_runtime.h>
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

__global__ void k_emtm_max(EmtmArgs a)
{
    const int p = blockIdx.y;
    if (p == a.ref) return;
    const long long nvox = (long long)a.nx * a.ny * a.nz;
    const float *d = a.dose + (size_t)p * nvox;
    const float *r = a.rho + (size_t)p * nvox;
    float m = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride)
        m = fmaxf(m, fmaxf(r[i] * d[i], 0.0f));
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(a.maxbits + p, __float_as_uint(m));
}

__global__ void k_emtm(EmtmArgs a)
{
    const int S = a.dvf4 ? a.phase : (int)blockIdx.y;
    if (S == a.ref) return;
    // the subvoxel-centre fractions (k + 1/2) / n of each axis, once per block
    __shared__ float s_frac[3][64];
    for (int t = threadIdx.x; t < 3 * 64; t += blockDim.x) {
        const int ax = t >> 6, k = t & 63;
        const int n = ax == 0 ? a.nsx : ax == 1 ? a.nsy : a.nsz;
        s_frac[ax][k] = k < n ? __fdiv_rn(__fadd_rn((float)k, 0.5f), (float)n) : 0.0f;
    }
    __syncthreads();
    const long long nvox = (long long)a.nx * a.ny * a.nz;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long pushed = 0, dropped = 0, pairs = 0;
    if (j < nvox) {
        const unsigned ju = (unsigned)j, row = ju / (unsigned)a.nx;      // nvox < 2^31
        const int jx = (int)(ju - row * (unsigned)a.nx);
        const int jy = (int)(row % (unsigned)a.ny);
        const int jz = (int)(row / (unsigned)a.ny);
        const float rho = a.rho[(size_t)S * nvox + j];
        const float dj = a.dose[(size_t)S * nvox + j];
        const int es = energy_shift(a.maxbits[S]);
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

__global__ void k_dvf4(const float *__restrict__ src, float4 *__restrict__ dst, long long nvox)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride)
        dst[i] = make_float4(src[i], src[nvox + i], src[2 * nvox + i], 0.0f);
}

__global__ void k_emtm_sum(EmtmArgs a)
{
    const long long nvox = (long long)a.nx * a.ny * a.nz;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
        double acc = (double)a.dose[(size_t)a.ref * nvox + i];
        for (int S = 0; S < a.n_phases; ++S) {
            if (S == a.ref) continue;
            const unsigned long long m = a.M[(size_t)S * nvox + i];
            if (m == 0) continue;
            // E / M back to Gy: times 2^(mass shift - energy shift), an exact
            // power of two built from its exponent bits
            const int k = kMassShift - energy_shift(a.maxbits[S]);
            const double q = div64((double)a.E[(size_t)S * nvox + i], (double)m);
            acc += (k > -1000 && k < 1000) ? q * __longlong_as_double((long long)(1023 + k) << 52) : ldexp(q, k);
        }
        if (a.mask && !a.mask[i]) acc = 0.0;
        a.accum[i] = (float)acc;
    }
}

}  // namespace dose
