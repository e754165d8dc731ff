// Host FP64 builder of the transport's lookup tables, stored as FP32.
//
// Model (project choices; Sec. 2.C of the paper names a class II condensed-
// history engine but prints no physics):
//   * Bethe mass stopping power of water with the full maximum energy
//     transfer, I = 75 eV, no shell/density/Barkas terms;
//   * CSDA range R(E) = integral from 0.5 MeV to E of dE'/S(E'), in mm of
//     water at 1 g/cm^3, and its inverse E(R);
//   * Bohr straggling variance per mm of water path,
//     K m_e c^2 (Z/A) (1 - beta^2/2)/(1 - beta^2) / 10;
//   * p v (MeV), from which the transport forms the Highland coefficient
//     (13.6 MeV / pv)^2 (pv is nearly linear in E, so it interpolates well);
//   * nuclear removal Sigma_w(E) = 0.0123 (1 - exp(-(E - 7)/20)) per cm above
//     7 MeV, stored per mm;
//   * HU -> (density, stopping-power ratio), piecewise linear.
// Integration here is composite Simpson on a fine sub-grid and inversion is
// bisection; results agree with an independent adaptive quadrature to far
// below FP32 resolution.
#include <cmath>
#include <vector>
#include "engine.cuh"

namespace dose {
namespace {

constexpr double K = 0.307075, ME = 0.51099895, MP = 938.27208816, ZA = 0.55509, I_EV = 75.0e-6;
constexpr double ECUT = 0.5;

double stopping_power(double e)   // MeV cm^2 / g
{
    const double gamma = 1.0 + e / MP;
    const double g2 = gamma * gamma;
    const double beta2 = 1.0 - 1.0 / g2;
    const double ratio = ME / MP;
    const double tmax = 2.0 * ME * beta2 * g2 / (1.0 + 2.0 * gamma * ratio + ratio * ratio);
    const double log_arg = 2.0 * ME * beta2 * g2 * tmax / (I_EV * I_EV);
    return K * ZA / beta2 * (0.5 * std::log(log_arg) - beta2);
}

// Simpson's rule of 1/S over [a, b] with m (even) panels, in mm of water.
double range_piece(double a, double b, int m)
{
    if (b <= a) return 0.0;
    const double h = (b - a) / m;
    double s = 1.0 / stopping_power(a) + 1.0 / stopping_power(b);
    for (int i = 1; i < m; ++i) s += (i % 2 ? 4.0 : 2.0) / stopping_power(a + i * h);
    return 10.0 * s * h / 3.0;
}

struct RangeTable {
    std::vector<double> node;   // R at E = ECUT + k * step
    double step = 1.0 / 64.0;
    RangeTable()
    {
        const int n = (int)((kEmax + 8.0 - ECUT) / step) + 2;
        node.resize(n);
        node[0] = 0.0;
        for (int k = 1; k < n; ++k)
            node[k] = node[k - 1] + range_piece(ECUT + (k - 1) * step, ECUT + k * step, 16);
    }
    double operator()(double e) const
    {
        if (e <= ECUT) return 0.0;
        int k = (int)((e - ECUT) / step);
        if (k >= (int)node.size() - 1) k = (int)node.size() - 2;
        const double ek = ECUT + k * step;
        return node[k] + range_piece(ek, e, 16);
    }
    double inverse(double r) const
    {
        if (r <= 0.0) return ECUT;
        double lo = ECUT, hi = kEmax + 8.0;
        for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; ++it) {
            const double mid = 0.5 * (lo + hi);
            if ((*this)(mid) < r) lo = mid; else hi = mid;
        }
        return 0.5 * (lo + hi);
    }
};

double calib(double hu, const double *y)
{
    static const double x[5] = {-1000.0, 0.0, 100.0, 1200.0, 3000.0};
    if (hu <= x[0]) return y[0];
    if (hu >= x[4]) return y[4];
    int k = 0;
    while (hu > x[k + 1]) ++k;
    return y[k] + (hu - x[k]) / (x[k + 1] - x[k]) * (y[k + 1] - y[k]);
}

}  // namespace

void build_tables(Tables *t, float *inv_ds)
{
    static const double rho_y[5] = {0.0012, 1.000, 1.100, 1.727, 2.753};
    static const double spr_y[5] = {0.00107, 1.000, 1.085, 1.640, 2.500};
    const RangeTable R;
    const double e_floor = ECUT;     // below the cut-off, tabulate the cut-off values
    for (int i = 0; i < kNE + 2; ++i) {
        const double e = std::fmin((double)i * kDE, (double)kEmax + kDE);
        const double ee = std::fmax(e, e_floor);
        const double gamma = 1.0 + ee / MP;
        const double bohr = K * ME * ZA * 0.5 * (gamma * gamma + 1.0) / 10.0;
        const double pv = ee * (ee + 2.0 * MP) / (ee + MP);
        const double sig = ee > 7.0 ? 0.0123 * (1.0 - std::exp(-(ee - 7.0) / 20.0)) / 10.0 : 0.0;
        t->re[i] = make_float4((float)R(e), (float)bohr, 0.0f, 0.0f);
        t->hs[i] = make_float4((float)pv, (float)sig, 0.0f, 0.0f);
    }
    const double ds = std::sqrt((double)kRmax) / kNR;
    for (int i = 0; i < kNR + 4; ++i) {
        const double r = (i * ds) * (i * ds);
        t->er[i] = make_float2((float)R.inverse(r), 0.0f);
    }
    // FP32 differences to the next entry (volatile: rounded as stored floats)
    for (int i = 0; i + 1 < kNE + 2; ++i) {
        volatile float rz = t->re[i + 1].x - t->re[i].x, rw = t->re[i + 1].y - t->re[i].y;
        volatile float hz = t->hs[i + 1].x - t->hs[i].x, hw = t->hs[i + 1].y - t->hs[i].y;
        t->re[i].z = rz; t->re[i].w = rw;
        t->hs[i].z = hz; t->hs[i].w = hw;
    }
    for (int i = 0; i + 1 < kNR + 4; ++i) {
        volatile float d = t->er[i + 1].x - t->er[i].x;
        t->er[i].y = d;
    }
    for (int i = 0; i < kNHU + 3; ++i) {
        const double hu = std::fmin((double)(kHuMin + i), (double)kHuMax);
        t->mat[i] = make_float2((float)calib(hu, rho_y), (float)calib(hu, spr_y));
    }
    *inv_ds = (float)(1.0 / ds);
}

}  // namespace dose
