// Delivery-timeline kernel (Sec. 2.B and App. A of Pepin et al.): integer-ns
// breathing clock and spot clock, one thread per field.  A spill crossing a
// phase boundary is split by time share (floor for each portion, the
// remainder to the last); gated delivery skips to the start of the next
// gate-on phase and adds the beam-discard time; each layer is painted
// `repaints` times.  All arithmetic is integer, so the subplans are exact.
#include <cuda_runtime.h>
#include "engine.cuh"
#include "kernels.h"

namespace dose {

namespace {
// floor(a b / w) with a b / w < 2^64
__device__ unsigned long long mul_div_floor(unsigned long long a, unsigned long long b,
                                            unsigned long long w)
{
    const unsigned long long lo = a * b, hi = __umul64hi(a, b);
    if (hi == 0) return lo / w;
    unsigned long long rem = hi, quo = 0;
    for (int i = 63; i >= 0; --i) {
        const unsigned long long carry = rem >> 63;
        rem = (rem << 1) | ((lo >> i) & 1ull);
        quo <<= 1;
        if (carry || rem >= w) { rem -= w; quo |= 1ull; }
    }
    return quo;
}

struct Clock {
    long long tph;
    unsigned long long p0, n;
    int gated, g0, g1;
    long long discard;
    __device__ unsigned phase(long long t) const
    {
        return (unsigned)((p0 + (unsigned long long)(t / tph)) % n);
    }
    __device__ bool on(unsigned ph) const
    {
        return !gated || ((int)ph >= g0 && (int)ph <= g1);
    }
    __device__ long long wait(long long t) const
    {
        while (!on(phase(t))) {
            const long long next = t / tph + 1;
            const long long ph_next = (long long)((p0 + (unsigned long long)next) % n);
            long long delta = ((long long)g0 - ph_next) % (long long)n;
            if (delta < 0) delta += (long long)n;
            t = (next + delta) * tph + discard;
        }
        return t;
    }
};
}  // namespace

__global__ void k_timeline(TimelineArgs a)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= a.n_fields) return;
    const int S = a.n_spots;
    Clock C;
    C.tph = a.tph;
    C.n = (unsigned long long)a.n_phases;
    C.gated = a.gated; C.g0 = a.gate_first; C.g1 = a.gate_last;
    C.discard = a.discard;
    if (a.start_phase >= 0) {
        C.p0 = (unsigned long long)a.start_phase;
    } else {
        const uint4 w = philox4x32_10(make_uint4((unsigned)f, 0u, 0u, 0u), (unsigned)a.seed,
                                      (unsigned)(a.seed >> 32));
        C.p0 = w.x % (unsigned)a.n_phases;
    }
    a.start_out[f] = (int)C.p0;
    const unsigned long long k = (unsigned long long)a.repaints;
    long long t = 0;
    bool delivered_any = false;
    int s = 0;
    while (s < S) {
        if (a.field[s] != f) { ++s; continue; }
        const int l0 = s;
        int l1 = s;
        for (int q = s + 1; q < S; ++q) {
            if (a.field[q] != f) continue;
            if (a.layer[q] != a.layer[l0]) break;
            l1 = q;
        }
        s = l1 + 1;
        bool layer_started = false;
        for (unsigned long long r = 0; r < k; ++r) {
            for (int q = l0; q <= l1; ++q) {
                if (a.field[q] != f) continue;
                const unsigned long long p = a.protons[q];
                unsigned long long w = p / k;
                if (r == k - 1) w += p % k;
                if (w == 0) continue;
                if (delivered_any) t += layer_started ? a.spot_switch : a.layer_switch;
                delivered_any = true;
                layer_started = true;
                const unsigned long long dur = mul_div_floor(w, 1000000000ull, a.rate);
                if (C.gated) t = C.wait(t);
                if (dur == 0) {
                    a.pp[(size_t)C.phase(t) * S + q] += w;
                    continue;
                }
                unsigned long long rem = dur, given = 0;
                while (rem > 0) {
                    if (C.gated) t = C.wait(t);
                    const long long seg = (t / C.tph + 1) * C.tph - t;
                    const unsigned long long d = rem < (unsigned long long)seg ? rem : (unsigned long long)seg;
                    const unsigned ph = C.phase(t);
                    t += (long long)d;
                    rem -= d;
                    const unsigned long long pj = rem > 0 ? mul_div_floor(w, d, dur) : w - given;
                    given += pj;
                    a.pp[(size_t)ph * S + q] += pj;
                }
            }
        }
    }
    a.field_end[f] = t;
}

}  // namespace dose
