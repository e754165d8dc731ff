// Dose-interpolation accumulation (Sec. 2.D.2, Eq. 3 of Pepin et al.) fused
// with the phase sum of Eq. 2.
//
//   k_dim  one thread per reference voxel i (x fastest, so a warp reads
//          consecutive voxels): for every source phase S != R, the voxel is
//          split into nsx x nsy x nsz subvoxels whose centres are carried to
//          S by the reference-to-source displacement field (trilinear
//          between the reference voxel centres), the dose of S is
//          interpolated trilinearly at each carried point, and the mean over
//          the subvoxels is D_i^S.  D_i = D_i^R + sum_S D_i^S, zero outside
//          the mask.  Both interpolations clamp to the edge beyond the
//          outermost voxel centres.
//
// A subvoxel centre sits at offset delta = (k + 1/2)/n - 1/2 from the voxel
// centre along each axis, inside the cell (i-1, i) when delta < 0 and
// (i, i+1) otherwise.  The subvoxels are therefore visited by octant: the
// eight field nodes of an octant's cell are loaded once (24 values) and
// every subvoxel of the octant is interpolated from registers.  The dose
// taps of the carried points are arbitrary and go through the L1 cache; the
// eight taps of the last cell are kept, since neighbouring subvoxels mostly
// land in the same cell of the source dose.
// Each phase's subvoxel sum is FP32 and the phase sum FP64; the pull needs
// no atomics, so the result does not depend on the launch.  A phase adds
// nothing to the reference voxels out of its reach (reach_box with mult 1,
// from k_reach over D != 0), which skip it.
#include <cuda_runtime.h>
#include <climits>
#include "engine.cuh"
#include "kernels.h"

namespace dose {

namespace {

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

}  // namespace

__global__ void __launch_bounds__(256, 3) k_dim(DimArgs a)
{
    const long long nvox = (long long)a.nx * a.ny * a.nz;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvox) return;
    const unsigned iu = (unsigned)i, row = iu / (unsigned)a.nx;     // nvox < 2^31
    const int ix = (int)(iu - row * (unsigned)a.nx);
    const int iy = (int)(row % (unsigned)a.ny);
    const int iz = (int)(row / (unsigned)a.ny);
    const int ns[3] = {a.nsx, a.nsy, a.nsz};
    const int ii[3] = {ix, iy, iz};
    const int nn[3] = {a.nx, a.ny, a.nz};
    const float inv_n[3] = {1.0f / (float)a.nsx, 1.0f / (float)a.nsy, 1.0f / (float)a.nsz};
    const float inv_nk = 1.0f / ((float)a.nsx * (float)a.nsy * (float)a.nsz);

    double acc = (double)a.dose[(size_t)a.ref * nvox + i];
    for (int S = 0; S < a.n_phases; ++S) {
        if (S == a.ref) continue;
        // out of reach of the phase's dose: every tap is zero
        const VoxBox b = reach_box(a.reach + (size_t)S * kReachWords, 1, a.nx, a.ny, a.nz, a.idx, a.idy, a.idz);
        if (ix < b.lo[0] || ix > b.hi[0] || iy < b.lo[1] || iy > b.hi[1] || iz < b.lo[2] || iz > b.hi[2]) continue;
        const float *ds = a.dose + (size_t)S * nvox;
        const float *dv = a.dvf ? a.dvf + (size_t)S * 3 * nvox : nullptr;
        float sum = 0.0f;
        int ck[3] = {INT_MIN, INT_MIN, INT_MIN};      // cell of the cached dose taps
        float cv[8];
        for (int oct = 0; oct < 8; ++oct) {
            // this octant's subvoxel index range and field cell, per axis
            int k0[3], k1[3], c0[3], c1[3];
            bool empty = false;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const bool up = (oct >> ax) & 1;
                const int half = ns[ax] >> 1;             // subvoxels with delta < 0
                k0[ax] = up ? half : 0;
                k1[ax] = up ? ns[ax] : half;
                empty |= k0[ax] >= k1[ax];
                const int lo = up ? ii[ax] : ii[ax] - 1;
                c0[ax] = min(max(lo, 0), nn[ax] - 1);
                c1[ax] = min(max(lo + 1, 0), nn[ax] - 1);
            }
            if (empty) continue;
            // the cell's eight field nodes (x fastest), mm -> voxels
            float u[3][8];
            if (dv) {
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    const size_t at = ((size_t)((cc & 4) ? c1[2] : c0[2]) * a.ny + ((cc & 2) ? c1[1] : c0[1])) * a.nx +
                                      ((cc & 1) ? c1[0] : c0[0]);
                    u[0][cc] = __ldg(dv + at) * a.idx;
                    u[1][cc] = __ldg(dv + nvox + at) * a.idy;
                    u[2][cc] = __ldg(dv + 2 * nvox + at) * a.idz;
                }
            }
            const bool upx = oct & 1, upy = (oct >> 1) & 1, upz = (oct >> 2) & 1;
            for (int kz = k0[2]; kz < k1[2]; ++kz) {
                const float dz = fmaf((float)kz + 0.5f, inv_n[2], -0.5f);       // delta
                const float fz = upz ? dz : 1.0f + dz;                          // in-cell fraction
                // field bilinear in (x, y) is done per subvoxel below; z first
                float uz[3][4];
                if (dv) {
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int q = 0; q < 4; ++q) uz[c][q] = lerpf(u[c][q], u[c][q + 4], fz);
                }
                const float qz = (float)iz + dz;
                for (int ky = k0[1]; ky < k1[1]; ++ky) {
                    const float dy = fmaf((float)ky + 0.5f, inv_n[1], -0.5f);
                    const float fy = upy ? dy : 1.0f + dy;
                    const float qy = (float)iy + dy;
                    for (int kx = k0[0]; kx < k1[0]; ++kx) {
                        const float dx = fmaf((float)kx + 0.5f, inv_n[0], -0.5f);
                        const float fx = upx ? dx : 1.0f + dx;
                        const float qx = (float)ix + dx;
                        float tx = qx, ty = qy, tz = qz;
                        if (dv) {
                            tx += lerpf(lerpf(uz[0][0], uz[0][1], fx), lerpf(uz[0][2], uz[0][3], fx), fy);
                            ty += lerpf(lerpf(uz[1][0], uz[1][1], fx), lerpf(uz[1][2], uz[1][3], fx), fy);
                            tz += lerpf(lerpf(uz[2][0], uz[2][1], fx), lerpf(uz[2][2], uz[2][3], fx), fy);
                        }
                        // neighbouring subvoxels usually land in the same cell: reuse its taps
                        const float gx = floorf(tx), gy = floorf(ty), gz = floorf(tz);
                        const int cx = (int)gx, cy = (int)gy, cz = (int)gz;
                        if (cx != ck[0] || cy != ck[1] || cz != ck[2]) {
                            ck[0] = cx; ck[1] = cy; ck[2] = cz;
                            const int x0 = min(max(cx, 0), a.nx - 1), x1 = min(max(cx + 1, 0), a.nx - 1);
                            const int y0 = min(max(cy, 0), a.ny - 1), y1 = min(max(cy + 1, 0), a.ny - 1);
                            const int z0 = min(max(cz, 0), a.nz - 1), z1 = min(max(cz + 1, 0), a.nz - 1);
                            const size_t r00 = ((size_t)z0 * a.ny + y0) * a.nx, r10 = ((size_t)z0 * a.ny + y1) * a.nx;
                            const size_t r01 = ((size_t)z1 * a.ny + y0) * a.nx, r11 = ((size_t)z1 * a.ny + y1) * a.nx;
                            cv[0] = __ldg(ds + r00 + x0); cv[1] = __ldg(ds + r00 + x1);
                            cv[2] = __ldg(ds + r10 + x0); cv[3] = __ldg(ds + r10 + x1);
                            cv[4] = __ldg(ds + r01 + x0); cv[5] = __ldg(ds + r01 + x1);
                            cv[6] = __ldg(ds + r11 + x0); cv[7] = __ldg(ds + r11 + x1);
                        }
                        const float hx = tx - gx, hy = ty - gy, hz = tz - gz;
                        sum += lerpf(lerpf(lerpf(cv[0], cv[1], hx), lerpf(cv[2], cv[3], hx), hy),
                                     lerpf(lerpf(cv[4], cv[5], hx), lerpf(cv[6], cv[7], hx), hy), hz);
                    }
                }
            }
        }
        acc += (double)(sum * inv_nk);
    }
    if (a.mask && !a.mask[i]) acc = 0.0;
    a.accum[i] = (float)acc;
}

}  // namespace dose
