// Delivery-timeline kernel (Sec. 2.B and App. A of Pepin et al.): integer-ns
// breathing clock and spot clock, one thread per (trial, field).
//
// Breathing: the clock starts at the beginning of phase p0 of cycle 0; cycle
// c lasts N t_c, t_c = floor(T_c / N), T_c = mu, or with sigma > 0
// max(N, mu + round(sigma Z_c)) where 2^21 Z_c is the Irwin-Hall sum of the
// twelve 21-bit fields of Philox blocks (f, c, 1, 0), (f, c, 2, 0) minus
// 6 (2^21 - 1) -- exact integers, so the phase lengths are reproducible.
//
// Spills: floor(w 1e9 / rate) ns each, split over the phase slots they span
// by time share (floor per portion, the remainder to the last).  Layers are
// painted `repaints` times (floor split, remainder last) or, with a cap m,
// until done with min(left, m) per spot and painting.
//   synchrotron = 0: switch times before every spill but a field's first;
//     gated delivery skips from a gate-off phase to the next gate_first
//     phase start and adds the discard.
//   synchrotron = 1 (App. A): fills.  A fill starts with a reset (the layer
//     switch; not for a field's first fill), a hold until the gate is on
//     (gated) and the beam discard; each layer takes a new fill; spills of
//     a fill are separated by the spot switch; a spill stops at the fill's
//     charge, its extraction time limit or a gate-off (floor(w elapsed /
//     duration) protons for a time cut) and the rest follows at the next
//     extraction start (after a hold and discard at a gate-off, in a new
//     fill otherwise).
// Uncertainty trials draw their parameters in the kernel (sample_trial).
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

__device__ __forceinline__ long long spill_ns(unsigned long long w, unsigned long long rate)
{
    return (long long)mul_div_floor(w, 1000000000ull, rate);
}

// 2^21 x (Irwin-Hall sum of twelve uniforms - 6) from blocks (a, b, c, 0), (a, b, c + 1, 0).
__device__ long long irwin_hall(unsigned long long seed, unsigned a, unsigned b, unsigned c)
{
    long long k = 0;
#pragma unroll
    for (unsigned blk = 0; blk < 2; ++blk) {
        const uint4 w = philox4x32_10(make_uint4(a, b, c + blk, 0u), (unsigned)seed, (unsigned)(seed >> 32));
        const unsigned long long lo = (unsigned long long)w.x | ((unsigned long long)w.y << 32);
        const unsigned long long hi = (unsigned long long)w.z | ((unsigned long long)w.w << 32);
        k += (long long)(lo & 0x1FFFFF) + (long long)((lo >> 21) & 0x1FFFFF) + (long long)((lo >> 42) & 0x1FFFFF);
        k += (long long)(((lo >> 63) | (hi << 1)) & 0x1FFFFF) + (long long)((hi >> 20) & 0x1FFFFF) +
             (long long)((hi >> 41) & 0x1FFFFF);
    }
    return k - 6ll * 0x1FFFFF;
}

// mean + round(sigma z / 2^21), half up (sigma < 2^38, |z| < 2^24: no overflow)
__device__ __forceinline__ long long gauss(long long mean, long long sigma, long long z)
{
    const long long num = sigma * z + (1ll << 20);
    return mean + (num >> 21);                     // arithmetic shift: floor
}

struct Clock {
    const dose_delivery *D;
    unsigned f;
    long long N, cyc_start, tph;
    unsigned long long cycle;
    long long s0 = 0, s1 = -1;                     // the last slot looked up: [s0, s1), phase ph
    unsigned ph = 0;

    __device__ long long cycle_tph(unsigned long long c) const
    {
        long long T = D->period_ns;
        if (D->period_sigma_ns > 0) {
            T = gauss(T, D->period_sigma_ns, irwin_hall(D->seed, f, (unsigned)c, 1u));
            if (T < N) T = N;
        }
        return T / N;
    }
    __device__ void sync(long long t)
    {
        while (t >= cyc_start + N * tph) {
            cyc_start += N * tph;
            ++cycle;
            tph = cycle_tph(cycle);
        }
    }
    // The clock moves forward, so most look-ups fall in the slot of the last
    // one and need no division.
    __device__ unsigned phase(long long t)
    {
        sync(t);
        if (t < s0 || t >= s1) {
            const long long k = (t - cyc_start) / tph;
            ph = (unsigned)k;
            s0 = cyc_start + k * tph;
            s1 = s0 + tph;
        }
        return ph;
    }
    __device__ long long slot_end(long long t) { phase(t); return s1; }
    __device__ bool on(unsigned ph) const
    {
        return !D->gated || ((int)ph >= D->gate_first && (int)ph <= D->gate_last);
    }
    __device__ long long hold(long long t)
    {
        while (!on(phase(t))) t = slot_end(t);
        return t;
    }
    __device__ long long off_after(long long t) const
    {
        Clock L = *this;                           // look ahead on a copy
        while (L.on(L.phase(t))) t = L.slot_end(t);
        return t;
    }
};

// Deliver w protons over [t, end) split at slot ends by time share.
__device__ void deposit(Clock &C, long long t, long long end, unsigned long long w,
                        unsigned long long *pp, int S, int q)
{
    if (w == 0) return;
    if (end <= t) { atomicAdd(pp + (size_t)C.phase(t) * S + q, w); return; }
    const unsigned long long dur = (unsigned long long)(end - t);
    unsigned long long given = 0;
    while (t < end) {
        const long long se = C.slot_end(t);
        const long long e = se < end ? se : end;
        const unsigned ph = C.phase(t);
        const unsigned long long pj = (e == end) ? w - given : mul_div_floor(w, (unsigned long long)(e - t), dur);
        given += pj;
        atomicAdd(pp + (size_t)ph * S + q, pj);
        t = e;
    }
}

constexpr int kMaxEmptyFills = 64;
constexpr long long kClockLimit = 1ll << 62;

struct Fill {
    bool in_fill = false;
    int fills = 0, spills = 0, empty = 0;
    long long ext_start = 0;
    unsigned long long left = 0, got = 0;
};

// Trial k's delivery: period from the discrete uniform set (word 0 of block
// (k, 0, 3, 0)), synchrotron parameters N(mean, sigma) (Irwin-Hall blocks
// (k, j, 4, 0), (k, j, 5, 0)), clamped at 0 (the rate at 1), trial seed
// seed + k 0x9E3779B97F4A7C15.
__device__ dose_delivery sample_trial(const dose_delivery &m, const dose_delivery_spread &s, unsigned long long k)
{
    dose_delivery d = m;
    if (s.period_max_ns > s.period_min_ns) {
        const unsigned long long n = (unsigned long long)((s.period_max_ns - s.period_min_ns) / s.period_step_ns) + 1;
        const uint4 w = philox4x32_10(make_uint4((unsigned)k, 0u, 3u, 0u), (unsigned)m.seed, (unsigned)(m.seed >> 32));
        d.period_ns = s.period_min_ns + (long long)(w.x % n) * s.period_step_ns;
    }
    const long long sig[6] = {s.spot_switch_sigma_ns, s.layer_switch_sigma_ns, s.discard_sigma_ns,
                              s.rate_sigma, s.fill_protons_sigma, s.extraction_limit_sigma_ns};
    long long v[6] = {m.spot_switch_ns, m.layer_switch_ns, m.discard_ns, (long long)m.rate_protons_per_s,
                      (long long)m.fill_protons, m.extraction_limit_ns};
    for (int j = 0; j < 6; ++j) {
        if (sig[j] == 0) continue;
        const long long g = gauss(v[j], sig[j], irwin_hall(m.seed, (unsigned)k, (unsigned)j, 4u));
        v[j] = g < 0 ? 0 : g;
    }
    d.spot_switch_ns = v[0];
    d.layer_switch_ns = v[1];
    d.discard_ns = v[2];
    d.rate_protons_per_s = (unsigned long long)(v[3] < 1 ? 1 : v[3]);
    d.fill_protons = (unsigned long long)v[4];
    d.extraction_limit_ns = v[5];
    d.seed = m.seed + k * 0x9E3779B97F4A7C15ull;
    return d;
}
}  // namespace

__global__ void k_timeline(const TimelineArgs *__restrict__ args)
{
    const TimelineArgs &a = args[blockIdx.x];
    // the plan's protons, layers and fields in shared memory (the walk below
    // reads them spot by spot)
    extern __shared__ unsigned long long s_prot[];
    const int S = a.n_spots;
    int *s_layer = reinterpret_cast<int *>(s_prot + S);
    unsigned char *s_field = reinterpret_cast<unsigned char *>(s_layer + S);
    for (int q = threadIdx.x; q < S; q += blockDim.x) {
        s_prot[q] = a.protons[q];
        s_layer[q] = a.layer[q];
        s_field[q] = (unsigned char)a.field[q];
    }
    __syncthreads();
    const int f = threadIdx.x;
    if (f >= a.n_fields) return;
    const dose_delivery D = a.spread ? sample_trial(a.d, *a.spread, a.trial) : a.d;
    if (f == 0 && a.used) *a.used = D;
    if (!delivery_ok(D)) {
        if (f == 0) *a.status = 1;
        return;
    }
    unsigned p0;
    if (D.start_phase >= 0) {
        p0 = (unsigned)D.start_phase;
    } else {
        const uint4 w = philox4x32_10(make_uint4((unsigned)f, 0u, 0u, 0u), (unsigned)D.seed, (unsigned)(D.seed >> 32));
        p0 = w.x % (unsigned)D.n_phases;
    }
    a.start_out[f] = (int)p0;
    Clock C;
    C.D = &D; C.f = (unsigned)f; C.N = D.n_phases; C.cycle = 0;
    C.tph = C.cycle_tph(0);
    C.cyc_start = -(long long)p0 * C.tph;
    const unsigned long long R = (unsigned long long)D.repaints, cap = D.max_protons_per_paint;
    Fill F;
    long long t = 0;
    bool delivered_any = false;
    int err = 0;
    int s = 0;
    while (s < S && !err) {
        if (s_field[s] != f) { ++s; continue; }
        const int l0 = s;
        int l1 = s;
        for (int q = s + 1; q < S; ++q) {
            if (s_field[q] != f) continue;
            if (s_layer[q] != s_layer[l0]) break;
            l1 = q;
        }
        s = l1 + 1;
        bool layer_started = false;
        F.in_fill = false;                               // a new energy takes a new fill
        for (unsigned long long r = 0; !err; ++r) {
            if (cap == 0 && r == R) break;
            bool any = false;
            for (int q = l0; q <= l1 && !err; ++q) {
                if (s_field[q] != f) continue;
                const unsigned long long p = s_prot[q];
                unsigned long long w;
                if (cap > 0) {
                    const unsigned long long done = r * cap;      // delivered by the earlier paintings
                    w = p > done ? min(p - done, cap) : 0ull;
                } else {
                    w = p / R;
                    if (r == R - 1) w += p % R;
                }
                if (w == 0) continue;
                any = true;
                if (D.synchrotron) {
                    bool first = true;
                    while (w > 0) {
                        if (!F.in_fill) {
                            if (F.fills > 0) {
                                F.empty = F.got ? 0 : F.empty + 1;
                                if (F.empty > kMaxEmptyFills) { err = 2; break; }
                                t += D.layer_switch_ns;
                            }
                            ++F.fills;
                            if (D.gated) t = C.hold(t);
                            t += D.discard_ns;
                            F.ext_start = t;
                            F.left = D.fill_protons;
                            F.in_fill = true;
                            F.spills = 0;
                            F.got = 0;
                        } else if (first && F.spills > 0) {
                            t += D.spot_switch_ns;
                        }
                        first = false;
                        const long long lim = D.extraction_limit_ns > 0 ? F.ext_start + D.extraction_limit_ns : LLONG_MAX;
                        if (D.gated && !C.on(C.phase(t))) {
                            const long long resume = C.hold(t) + D.discard_ns;
                            if (resume >= lim) {                 // the fill expires while held
                                if (t < lim) t = lim;
                                F.in_fill = false;
                                continue;
                            }
                            t = resume;
                        }
                        if (t >= lim) { F.in_fill = false; continue; }
                        if (t > kClockLimit) { err = 3; break; }
                        unsigned long long part = w;
                        if (D.fill_protons > 0 && F.left < part) part = F.left;
                        const long long dur = spill_ns(part, D.rate_protons_per_s);
                        long long end = t + dur;
                        int cut = 0;                             // 1: time limit, 2: gate-off
                        if (end > lim) { end = lim; cut = 1; }
                        if (D.gated) {
                            const long long off = C.off_after(t);
                            if (end > off) { end = off; cut = 2; }
                        }
                        const unsigned long long now =
                            cut ? mul_div_floor(part, (unsigned long long)(end - t), (unsigned long long)dur) : part;
                        deposit(C, t, end, now, a.pp, S, q);
                        t = end;
                        w -= now;
                        F.got += now;
                        ++F.spills;
                        if (D.fill_protons > 0) F.left -= now;
                        if (cut == 1 || (D.fill_protons > 0 && F.left == 0)) F.in_fill = false;
                    }
                    continue;
                }
                if (delivered_any) t += layer_started ? D.spot_switch_ns : D.layer_switch_ns;
                delivered_any = true;
                layer_started = true;
                if (t > kClockLimit) { err = 3; break; }
                const long long dur = spill_ns(w, D.rate_protons_per_s);
                if (D.gated && !C.on(C.phase(t))) t = C.hold(t) + D.discard_ns;
                if (dur == 0) {
                    atomicAdd(a.pp + (size_t)C.phase(t) * S + q, w);
                    continue;
                }
                long long rem = dur;
                unsigned long long given = 0;
                while (rem > 0) {
                    if (D.gated && !C.on(C.phase(t))) t = C.hold(t) + D.discard_ns;
                    const long long seg = C.slot_end(t) - t;
                    const long long d = rem < seg ? rem : seg;
                    const unsigned ph = C.phase(t);
                    t += d;
                    rem -= d;
                    const unsigned long long pj = rem > 0 ? mul_div_floor(w, (unsigned long long)d, (unsigned long long)dur)
                                                          : w - given;
                    given += pj;
                    atomicAdd(a.pp + (size_t)ph * S + q, pj);
                }
            }
            if (cap > 0 && !any) break;
        }
    }
    a.field_end[f] = t;
    if (err) atomicMax(a.status, err);
}

}  // namespace dose
