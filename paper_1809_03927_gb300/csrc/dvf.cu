// Decoding a deformable registration's vector grid onto the CT grid
// (App. B, Eqs. 7-8 of Pepin et al.), the first of the paper's two
// accumulation-side GPU steps.
//
//   k_dvf_grid      one thread per registration-grid voxel (i, j, k): its
//                   position r0 = start + i dX U + j dY V + k dZ W, W = U x V
//                   (Eq. 8), and mapped position r_f = M_post (M_pre r0 +
//                   Delta) (Eq. 7), stored as the grid displacement
//                   e = r_f - r0 = (R_post R_pre - I) r0 + R_post (t_pre +
//                   Delta) + t_post, which keeps FP32 precision where the
//                   rigid parts are the identity (the 4DCT case).
//   k_dvf_resample  one thread per CT voxel: the continuous grid index of
//                   its centre p, (U.(p - start)/dX, V.(p - start)/dY,
//                   W.(p - start)/dZ); inside the hull of grid voxel centres
//                   the displacement is the trilinear interpolant of e
//                   (= interpolated r_f - p, since r0 is affine in the
//                   index), outside it is 0 and the voxel leaves the mask.
//
// The inside test is an integer decision taken in single precision with the
// rounding order written out (no contraction), so it is reproducible.
#include <cuda_runtime.h>
#include "engine.cuh"
#include "kernels.h"

namespace dose {

__global__ void k_dvf_grid(DvfArgs a)
{
    const long long ng = (long long)a.gn[0] * a.gn[1] * a.gn[2];
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    // grid and CT voxel counts are below 2^31: 32-bit index arithmetic
    const unsigned gu = (unsigned)g, row = gu / (unsigned)a.gn[0];
    const int i = (int)(gu - row * (unsigned)a.gn[0]);
    const int j = (int)(row % (unsigned)a.gn[1]);
    const int k = (int)(row / (unsigned)a.gn[1]);
    const float si = i * a.sp[0], sj = j * a.sp[1], sk = k * a.sp[2];
    float r0[3], d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        r0[c] = fmaf(sk, a.W[c], fmaf(sj, a.V[c], fmaf(si, a.U[c], a.start[c])));
        d[c] = a.delta[3 * g + c] + a.pre[4 * c + 3];                   // t_pre + Delta
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        // (R_post R_pre - I) r0 + R_post (t_pre + Delta) + t_post
        float e = a.post[4 * c + 3];
#pragma unroll
        for (int m = 0; m < 3; ++m) e = fmaf(a.RR[3 * c + m], r0[m], fmaf(a.post[4 * c + m], d[m], e));
        a.e[c * ng + g] = e;
    }
}

__global__ void k_dvf_resample(DvfArgs a)
{
    const long long nvox = (long long)a.n[0] * a.n[1] * a.n[2];
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const unsigned vu = (unsigned)v, row = vu / (unsigned)a.n[0];
    const int ii[3] = {(int)(vu - row * (unsigned)a.n[0]), (int)(row % (unsigned)a.n[1]), (int)(row / (unsigned)a.n[1])};
    // W = U x V in the decision's precision and order
    const float Wf[3] = {__fsub_rn(__fmul_rn(a.U[1], a.V[2]), __fmul_rn(a.U[2], a.V[1])),
                         __fsub_rn(__fmul_rn(a.U[2], a.V[0]), __fmul_rn(a.U[0], a.V[2])),
                         __fsub_rn(__fmul_rn(a.U[0], a.V[1]), __fmul_rn(a.U[1], a.V[0]))};
    float rel[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float p = __fadd_rn(a.origin[c], __fmul_rn(__fadd_rn((float)ii[c], 0.5f), a.d[c]));
        rel[c] = __fsub_rn(p, a.start[c]);
    }
    const float *axes[3] = {a.U, a.V, Wf};
    float q[3];
    bool in = true;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float *u = axes[ax];
        const float dot = __fadd_rn(__fadd_rn(__fmul_rn(u[0], rel[0]), __fmul_rn(u[1], rel[1])),
                                    __fmul_rn(u[2], rel[2]));
        q[ax] = __fdiv_rn(dot, a.sp[ax]);
        in = in && q[ax] >= 0.0f && q[ax] <= (float)(a.gn[ax] - 1);
    }
    if (!in) {
        a.out[v] = 0.0f;
        a.out[nvox + v] = 0.0f;
        a.out[2 * nvox + v] = 0.0f;
        if (a.mask) a.mask[v] = 0;
        return;
    }
    int lo[3], hi[3];
    float f[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float fl = floorf(q[ax]);
        f[ax] = q[ax] - fl;
        lo[ax] = (int)fl;
        hi[ax] = min(lo[ax] + 1, a.gn[ax] - 1);
    }
    const long long ng = (long long)a.gn[0] * a.gn[1] * a.gn[2];
    const long long r00 = ((long long)lo[2] * a.gn[1] + lo[1]) * a.gn[0];
    const long long r10 = ((long long)lo[2] * a.gn[1] + hi[1]) * a.gn[0];
    const long long r01 = ((long long)hi[2] * a.gn[1] + lo[1]) * a.gn[0];
    const long long r11 = ((long long)hi[2] * a.gn[1] + hi[1]) * a.gn[0];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float *e = a.e + c * ng;
        auto lx = [&](long long r) { const float x0 = __ldg(e + r + lo[0]); return fmaf(f[0], __ldg(e + r + hi[0]) - x0, x0); };
        const float c00 = lx(r00), c10 = lx(r10), c01 = lx(r01), c11 = lx(r11);
        const float c0 = fmaf(f[1], c10 - c00, c00), c1 = fmaf(f[1], c11 - c01, c01);
        a.out[c * nvox + v] = fmaf(f[2], c1 - c0, c0);
    }
}

}  // namespace dose
