/*
 * FP64 CPU oracle of the Monte Carlo proton dose engine of the 4D-dose
 * calculator (Pepin et al., arXiv:1809.03927) and of its two companion
 * stages: the delivery timeline and the energy/mass-transfer accumulation.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * legs of the benchmark (cpu_baseline and the reference arm) load this
 * library.  The CUDA product path never links, loads or calls it.  This
 * file includes no project header and shares no table, constant generator
 * or helper with the CUDA path; both follow the same written model.
 *
 * The paper (Sec. 2.C) names the engine "class II condensed-history proton
 * transport" and says the MC converts HU to density, but prints no physics.
 * The model written out here is the project's: piecewise-linear HU
 * calibration, Bethe water stopping power (I = 75 eV) with CSDA range,
 * Highland multiple scattering in its cumulative-thickness form, Bohr
 * straggling and non-elastic nuclear removal with a fixed local-deposit
 * fraction.  Every function below says which passage or definition it
 * follows and what pins it:
 *
 *   or_philox4x32_10   Salmon et al., SC'11 (the cuRAND generator named in
 *                      Sec. 2.B, footnote b).  Pinned: published
 *                      known-answer vectors.
 *   or_rho, or_spr     Sec. 2.C (HU -> density).  Pinned: water (HU 0) is
 *                      exactly 1, air (HU -1000) is 0.0012 g/cm^3.
 *   or_bethe_sw        Bethe formula with full T_max.  Pinned: Bragg-Kleeman
 *                      rule (Bortfeld 1997) within 2 %.
 *   or_range, or_energy_from_range
 *                      CSDA range = integral of 1/S.  Pinned: independent
 *                      adaptive quadrature; R(E(R)) = R.
 *   or_allocate        Sec. 1 / 2.A (spots carry weights).  Pinned: brute
 *                      force on small cases, sum and bound invariants.
 *   or_transport       Sec. 2.C.  Pinned: CSDA range, range scaling with
 *                      SPR, R80, Fermi-Eyges lateral sigma, primary fluence,
 *                      energy balance, one-step moment checks.
 *   or_normalise       Sec. 2.C (dose and density outputs), Eq. 4 (E = M D).
 *                      Pinned: hand-worked unit conversion.
 *   or_timeline        Sec. 2.B, App. A.  Pinned: invariants (protons
 *                      conserved, clock total), the one-phase test of
 *                      Sec. 2.E, hand-worked examples (simple clock,
 *                      synchrotron fills, charge and time limits, gate
 *                      holds, capped repainting), the synchrotron model
 *                      reducing to the simple clock without limits, the
 *                      moments and bounds of the breathing deviates.
 *   or_trial_delivery  Sec. 2.B (the 25 uncertainty trials).  Pinned:
 *                      discrete-uniform periods, Gaussian moments.
 *   or_emtm            Sec. 2.D.2, Eqs. 2, 4-6, in FP64, with bounds for
 *                      points on cell faces.  Pinned: identity-DVF test of
 *                      Sec. 2.E, integer and half-voxel translations,
 *                      energy and mass conservation, the mask, convergence
 *                      in n, agreement with the DIM for inverse whole-voxel
 *                      shifts.
 *   or_dvf_decode      App. B, Eqs. 7-8, and the DICOM rule that positions
 *                      between grid voxels interpolate trilinearly; FP64,
 *                      with a flag for voxels on the hull faces.  Pinned:
 *                      uniform and affine translations (exact under
 *                      trilinear interpolation), rotated grid axes, the
 *                      depth axis W = U x V, rigid pre/post transforms, the
 *                      grid-hull mask.
 *   or_dim             Sec. 2.D.2, Eqs. 2-3.  Pinned: identity at n = 1,
 *                      exactness of trilinear interpolation on linear dose
 *                      and displacement fields, the interpolation error of a
 *                      quadratic dose in closed form, integer translation
 *                      and the direction of the field.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- physical constants (standard values; the paper gives none) -------- */
#define OR_K        0.307075         /* MeV cm^2 / mol                       */
#define OR_ME       0.51099895       /* electron rest energy, MeV            */
#define OR_MP       938.27208816     /* proton rest energy, MeV              */
#define OR_ZA       0.55509          /* water Z/A                            */
#define OR_I        75.0e-6          /* water mean excitation energy, MeV    */
#define OR_X0_MM    360.8            /* water radiation length 36.08 g/cm^2  */
#define OR_MEV_J    1.602176634e-13  /* J per MeV                            */
/* ---- transport model parameters (project choices) ---------------------- */
#define OR_ECUT     0.5              /* MeV: below this, deposit and stop    */
#define OR_FSTEP    0.25             /* step <= 0.25 x residual range        */
#define OR_SMIN     0.01             /* mm: minimum physics step             */
#define OR_SIG_INF  0.0123           /* 1/cm, nuclear Sigma_w at high energy */
#define OR_E_TH     7.0              /* MeV, nuclear threshold               */
#define OR_E_S      20.0             /* MeV, nuclear rise scale              */
#define OR_FLOC     0.6              /* local-deposit fraction at removal    */
#define OR_HL_A     13.6             /* Highland, MeV                        */
#define OR_HL_B     0.038            /* Highland log coefficient             */

#define OR_OK        0
#define OR_EINVAL   -1
#define OR_ENOMEM   -2
#define OR_ESTEP    -5

/* ======================================================================= */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).                      */
/* Round: two 32x32->64 products of counter words 0 and 2 with the         */
/* multipliers, outputs permuted and xor-ed with the key; the key gets a   */
/* Weyl increment between rounds.                                          */
/* ======================================================================= */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The random stream of history h (stream id st, 64-bit seed): block b is
 * Philox4x32-10 of counter (b, h_lo, h_hi, st) under key (seed_lo, seed_hi).
 * A block's 128 bits, read as one little-endian integer, give six 21-bit
 * integers k_i = bits [21 i, 21 i + 21), i = 0..5, and the uniforms
 * u_i = (k_i + 1/2) / 2^21, all in (0, 1) and exact in binary floating point.
 * Block 0 is the history's birth block, block k + 1 serves step k.          */
void or_block_uniforms(uint64_t seed, uint64_t h, uint32_t stream,
                       uint32_t block, double u[6])
{
    uint32_t ctr[4] = { block, (uint32_t)h, (uint32_t)(h >> 32), stream };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    unsigned __int128 v = (unsigned __int128)w[0] | ((unsigned __int128)w[1] << 32) |
                          ((unsigned __int128)w[2] << 64) | ((unsigned __int128)w[3] << 96);
    for (int i = 0; i < 6; ++i) {
        uint32_t k = (uint32_t)((v >> (21 * i)) & 0x1FFFFFu);
        u[i] = ((double)k + 0.5) / 2097152.0;
    }
}

/* Box-Muller: a pair of independent standard normals from two uniforms.    */
static void or_box_muller(double ua, double ub, double *z0, double *z1)
{
    const double two_pi = 6.283185307179586476925286766559;
    double r = sqrt(-2.0 * log(ua));
    *z0 = r * cos(two_pi * ub);
    *z1 = r * sin(two_pi * ub);
}

/* ======================================================================= */
/* HU -> mass density and stopping-power ratio (Sec. 2.C: the MC converts  */
/* Hounsfield units to density).  Piecewise linear through the project's   */
/* calibration points, HU clamped to [-1000, 3000].                        */
/* ======================================================================= */
static const double OR_CAL_HU[5]  = { -1000.0, 0.0, 100.0, 1200.0, 3000.0 };
static const double OR_CAL_RHO[5] = { 0.0012, 1.000, 1.100, 1.727, 2.753 };
static const double OR_CAL_SPR[5] = { 0.00107, 1.000, 1.085, 1.640, 2.500 };

static double or_piecewise(double hu, const double *y)
{
    if (hu <= OR_CAL_HU[0]) return y[0];
    if (hu >= OR_CAL_HU[4]) return y[4];
    int k = 0;
    while (!(hu >= OR_CAL_HU[k] && hu <= OR_CAL_HU[k + 1])) ++k;
    double t = (hu - OR_CAL_HU[k]) / (OR_CAL_HU[k + 1] - OR_CAL_HU[k]);
    return y[k] + t * (y[k + 1] - y[k]);
}
double or_rho(int hu) { return or_piecewise((double)hu, OR_CAL_RHO); }
double or_spr(int hu) { return or_piecewise((double)hu, OR_CAL_SPR); }

/* ======================================================================= */
/* Bethe mass stopping power of water, MeV cm^2/g, with the full maximum   */
/* energy transfer and no shell, density-effect or Barkas terms:           */
/*   S = K (Z/A) / beta^2 [ 1/2 ln(2 me beta^2 gamma^2 Tmax / I^2) - beta^2 ] */
/*   Tmax = 2 me beta^2 gamma^2 / (1 + 2 gamma me/mp + (me/mp)^2)          */
/* ======================================================================= */
double or_bethe_sw(double E)
{
    double gam = 1.0 + E / OR_MP;
    double bg2 = gam * gam - 1.0;              /* beta^2 gamma^2 */
    double b2 = bg2 / (gam * gam);
    double r = OR_ME / OR_MP;
    double tmax = 2.0 * OR_ME * bg2 / (1.0 + 2.0 * gam * r + r * r);
    double arg = 2.0 * OR_ME * bg2 * tmax / (OR_I * OR_I);
    return OR_K * OR_ZA / b2 * (0.5 * log(arg) - b2);
}

/* ---- CSDA range R(E) = integral_{Ecut}^{E} dE'/S(E') --------------------
 * Cumulative integrals on nodes E_k = Ecut + k h (h = 0.01 MeV) with an
 * n-point Gauss-Legendre rule per interval; R(E) between nodes adds the
 * same rule over [E_k, E].  Ranges are returned in mm of water (1 g/cm^3). */
#define OR_RH      0.01
#define OR_RNODES  26001                 /* up to Ecut + 260 MeV */
#define OR_GLN     4
static double or_gl_x[OR_GLN], or_gl_w[OR_GLN];
static double or_rcum[OR_RNODES];
static int or_tables_ready = 0;

/* Gauss-Legendre nodes/weights on [-1, 1] by Newton on P_n (three-term
 * recurrence), the textbook construction.                                  */
static void or_gauss_legendre(int n, double *x, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = cos(pi * (i + 0.75) / (n + 0.5));
        double pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2; p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z;
            z = z1 - p1 / pp;
            if (fabs(z - z1) < 1e-15) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

static double or_gl_inv_s(double a, double b)
{
    double c = 0.5 * (a + b), hw = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < OR_GLN; ++i) s += or_gl_w[i] / or_bethe_sw(c + hw * or_gl_x[i]);
    return s * hw;                       /* g/cm^2 */
}

void or_init_tables(void)
{
    if (or_tables_ready) return;
    or_gauss_legendre(OR_GLN, or_gl_x, or_gl_w);
    or_rcum[0] = 0.0;
    for (int k = 1; k < OR_RNODES; ++k) {
        double a = OR_ECUT + (k - 1) * OR_RH, b = OR_ECUT + k * OR_RH;
        or_rcum[k] = or_rcum[k - 1] + 10.0 * or_gl_inv_s(a, b);   /* mm */
    }
    or_tables_ready = 1;
}

double or_range(double E)
{
    if (E <= OR_ECUT) return 0.0;
    double x = (E - OR_ECUT) / OR_RH;
    int k = (int)floor(x);
    if (k >= OR_RNODES - 1) k = OR_RNODES - 2;
    double Ek = OR_ECUT + k * OR_RH;
    return or_rcum[k] + 10.0 * or_gl_inv_s(Ek, E);
}

/* Inverse of the range: bisection over the node table, then safeguarded
 * Newton (dR/dE = 1/S) to full double precision.                          */
double or_energy_from_range(double R)
{
    if (R <= 0.0) return OR_ECUT;
    int lo = 0, hi = OR_RNODES - 1;
    if (R >= or_rcum[hi]) return OR_ECUT + hi * OR_RH;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (or_rcum[mid] <= R) lo = mid; else hi = mid;
    }
    double a = OR_ECUT + lo * OR_RH, b = OR_ECUT + hi * OR_RH;
    double E = a + (R - or_rcum[lo]) / (or_rcum[hi] - or_rcum[lo]) * (b - a);
    for (int it = 0; it < 60; ++it) {
        double f = or_range(E) - R;
        if (f > 0.0) b = E; else a = E;
        double En = E - f * or_bethe_sw(E) / 10.0;
        if (fabs(En - E) <= 1e-13 * E) { E = En; break; }
        if (!(En >= a && En <= b)) En = 0.5 * (a + b);
        E = En;
    }
    return E;
}

/* Nuclear removal cross-section per water-equivalent length, 1/cm.         */
double or_sigma_nuc(double E)
{
    if (E <= OR_E_TH) return 0.0;
    return OR_SIG_INF * (1.0 - exp(-(E - OR_E_TH) / OR_E_S));
}

/* Highland cumulative function g(u) = u (1 + 0.038 ln u)^2, g(0) = 0.       */
static double or_highland_g(double u)
{
    if (u <= 0.0) return 0.0;
    double t = 1.0 + OR_HL_B * log(u);
    return u * t * t;
}

/* p v (MeV) of a proton of kinetic energy E: E (E + 2 mp) / (E + mp).     */
double or_pv(double E) { return E * (E + 2.0 * OR_MP) / (E + OR_MP); }

/* ---- pieces of one condensed-history step, shared by the transport and by
 * the single-step functions exposed for the pins ------------------------ */

/* CSDA over a water-equivalent path sw (mm) from energy E with residual
 * range R0: end energy E(R0 - sw) and the step-mean energy (E + E1)/2.     */
static void or_csda(double E, double R0, double sw, double *E1c, double *Emean)
{
    *E1c = or_energy_from_range(R0 - sw);
    *Emean = 0.5 * (E + *E1c);
}

/* Bohr straggling variance (MeV^2) over a water-equivalent path sw (mm):
 * K me (Z/A) sw[cm] (1 - beta^2/2)/(1 - beta^2), beta at the step start;
 * (1 - beta^2/2)/(1 - beta^2) = (gamma^2 + 1)/2.                          */
double or_bohr_var(double E, double sw_mm)
{
    double gam = 1.0 + E / OR_MP;
    return OR_K * OR_ME * OR_ZA * (sw_mm / 10.0) * 0.5 * (gam * gam + 1.0);
}

/* Energy loss of a step whose mean (CSDA) loss is m and whose Bohr
 * variance is v, from the standard normal z: lognormal with exactly that
 * mean and variance,
 *   dE = m exp(sig z - sig^2 / 2),  sig^2 = ln(1 + v / m^2),
 * so E[dE] = m and Var[dE] = m^2 (exp(sig^2) - 1) = v for every step length:
 * the moments of the loss over a path do not depend on how the path is cut
 * into steps (a Gaussian cut at zero or at +-m would lose variance on thin
 * steps, where sqrt(v) >> m).  The loss is never negative and, like the
 * loss in a thin absorber, skewed to high values; for thick steps
 * (v << m^2) it tends to the Gaussian.  A step without mean loss loses
 * nothing.                                                                 */
static double or_straggle_loss(double m, double v, double z)
{
    if (!(m > 0.0) || !(v > 0.0)) return m;
    double s2 = log1p(v / (m * m));
    return m * exp(sqrt(s2) * z - 0.5 * s2);
}

/* Highland variance of the projected angle over radiation thickness
 * [u0, u0 + du]: (13.6 / pv)^2 (g(u0 + du) - g(u0)), pv at energy E.      */
double or_highland_theta2(double E, double u0, double du)
{
    double k = OR_HL_A / or_pv(E);
    return k * k * (or_highland_g(u0 + du) - or_highland_g(u0));
}

/* Correlated lateral displacement and angle in one transverse plane over a
 * step s: y = s theta0 (z1/sqrt(12) + z2/2), theta = theta0 z2 (the PDG
 * Passage-of-particles form).                                             */
static void or_mcs_plane(double s, double th0, double z1, double z2, double *y, double *t)
{
    *y = s * th0 * (z1 / sqrt(12.0) + 0.5 * z2);
    *t = th0 * z2;
}

/* ======================================================================= */
/* Histories per spot: proportional to the spot's protons, floor plus      */
/* largest remainder; equal remainders go to the lower spot index.         */
/* ======================================================================= */
typedef struct { uint64_t rem; int64_t idx; } or_rem_t;

static int or_rem_cmp(const void *a, const void *b)
{
    const or_rem_t *x = (const or_rem_t *)a, *y = (const or_rem_t *)b;
    if (x->rem != y->rem) return x->rem > y->rem ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

int or_allocate(int64_t n_spots, const uint64_t *protons, uint64_t n_hist,
                uint64_t *n_out)
{
    if (n_spots <= 0) return OR_EINVAL;
    unsigned __int128 W = 0;
    for (int64_t s = 0; s < n_spots; ++s) W += protons[s];
    if (W == 0 || W > (unsigned __int128)UINT64_MAX) return OR_EINVAL;
    or_rem_t *r = (or_rem_t *)malloc(sizeof(or_rem_t) * (size_t)n_spots);
    if (!r) return OR_ENOMEM;
    uint64_t assigned = 0;
    for (int64_t s = 0; s < n_spots; ++s) {
        unsigned __int128 q = (unsigned __int128)n_hist * protons[s];
        n_out[s] = (uint64_t)(q / W);
        r[s].rem = (uint64_t)(q % W);
        r[s].idx = s;
        assigned += n_out[s];
    }
    uint64_t left = n_hist - assigned;
    qsort(r, (size_t)n_spots, sizeof(or_rem_t), or_rem_cmp);
    for (uint64_t i = 0; i < left; ++i) n_out[r[i].idx] += 1;
    free(r);
    return OR_OK;
}

/* ======================================================================= */
/* Transport (Sec. 2.C: class II condensed history).                       */
/* ======================================================================= */
typedef struct {
    /* grid: voxel (i,j,k) covers [i dx, (i+1) dx) x ... in grid mm; x fastest */
    int32_t n[3];
    double d[3];
    double origin[3];            /* patient-frame mm of the grid corner */
    const int16_t *hu;
    int32_t beam_axis;           /* 0, 1, 2 */
    int32_t beam_sign;           /* +1 or -1 */
    /* plan: spot lateral coordinates are the patient-frame coordinates on
       the two non-beam axes, lower axis first */
    int64_t n_spots;
    const double *spot_x, *spot_y, *spot_e, *spot_sigma;
    const uint64_t *spot_protons;
    /* run */
    uint64_t n_hist;             /* histories of the whole run */
    uint64_t hist_begin, hist_end;
    uint64_t seed;
    uint32_t stream;
    uint32_t physics;            /* bit0 straggling, bit1 MCS, bit2 nuclear */
    double spr_scale;
    double shift[3];             /* patient displacement, mm */
    int64_t max_steps;
    int32_t nthreads;
    /* diagnostics, depth measured from the upstream face along the beam */
    int32_t n_depth_bins;
    double depth_bin_mm;
    int32_t n_planes;
    double plane_mm;             /* plane k at depth (k + 1) plane_mm */
    /* run only the histories h of [hist_begin, hist_end) with
       h mod batch_count == batch_index (batch_count 0 or 1: all)          */
    uint64_t batch_count, batch_index;
} or_run_params;

typedef struct {
    double *edep;                /* nvox, MeV x history weight */
    double *depth_dose;          /* n_depth_bins or NULL */
    double *plane_w;             /* n_planes: weight of primaries crossing */
    double *plane_m1;            /* 2 x n_planes: sum w x (lateral axes) */
    double *plane_m2;            /* 2 x n_planes: sum w x^2 */
    double ledger[4];            /* deposited, escaped, removed, incident */
    uint64_t steps;
    uint64_t histories;
    int32_t status;
    double end_depth[3];         /* sum w z_end, sum w, sum w z_end^2 over
                                    histories that stop by running out of
                                    energy */
} or_run_out;

#define OR_PHYS_STRAG 1u
#define OR_PHYS_MCS   2u
#define OR_PHYS_NUC   4u

typedef struct {
    double *edep, *depth, *pw, *pm1, *pm2;
    double ledger[4];
    uint64_t steps;
    int32_t status;
    double end_depth[3];
} or_acc;

static void or_depth_spread(const or_run_params *P, or_acc *A, double z0,
                            double z1, double e)
{
    if (!A->depth || e == 0.0) return;
    double a = z0 < z1 ? z0 : z1, b = z0 < z1 ? z1 : z0;
    double w = P->depth_bin_mm;
    if (b - a < 1e-12) {
        int k = (int)floor(a / w);
        if (k >= 0 && k < P->n_depth_bins) A->depth[k] += e;
        return;
    }
    int ka = (int)floor(a / w), kb = (int)floor(b / w);
    for (int k = ka; k <= kb; ++k) {
        double lo = k * w > a ? k * w : a;
        double hi = (k + 1) * w < b ? (k + 1) * w : b;
        if (hi > lo && k >= 0 && k < P->n_depth_bins)
            A->depth[k] += e * (hi - lo) / (b - a);
    }
}

static double or_depth_of(const or_run_params *P, const double *p)
{
    int a = P->beam_axis;
    return P->beam_sign > 0 ? p[a] : P->n[a] * P->d[a] - p[a];
}

static void or_planes(const or_run_params *P, or_acc *A, const double *p0,
                      const double *p1, double w)
{
    if (!A->pw) return;
    int a = P->beam_axis, b = (a == 0) ? 1 : 0, c = (a == 2) ? 1 : 2;
    double z0 = or_depth_of(P, p0), z1 = or_depth_of(P, p1);
    if (z1 <= z0) return;
    int k0 = (int)floor(z0 / P->plane_mm);          /* planes with z0 < zk <= z1 */
    for (int k = k0; k < P->n_planes; ++k) {
        double zk = (k + 1) * P->plane_mm;
        if (zk <= z0) continue;
        if (zk > z1) break;
        double t = (zk - z0) / (z1 - z0);
        double xb = p0[b] + t * (p1[b] - p0[b]);
        double xc = p0[c] + t * (p1[c] - p0[c]);
        A->pw[k] += w;
        A->pm1[k] += w * xb;  A->pm1[P->n_planes + k] += w * xc;
        A->pm2[k] += w * xb * xb;  A->pm2[P->n_planes + k] += w * xc * xc;
    }
}

/* Orthonormal frame (e1, e2) perpendicular to unit vector d: the branch-free
 * construction of Duff et al., "Building an Orthonormal Basis, Revisited",
 * JCGT 6(1), 2017.                                                          */
void or_frame(const double *d, double *e1, double *e2)
{
    double sg = d[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + d[2]);
    double b = d[0] * d[1] * a;
    e1[0] = 1.0 + sg * d[0] * d[0] * a; e1[1] = sg * b; e1[2] = -sg * d[0];
    e2[0] = b; e2[1] = sg + d[1] * d[1] * a; e2[2] = -d[1];
}

/* One history.  Returns 0, or OR_ESTEP if the step limit was hit.           */
static void or_history(const or_run_params *P, const uint64_t *prefix,
                       const double *wts, uint64_t h, or_acc *A)
{
    /* spot of history h: prefix[s] <= h < prefix[s+1] */
    int64_t lo = 0, hi = P->n_spots;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (prefix[mid] <= h) lo = mid; else hi = mid;
    }
    int64_t s = lo;
    double w = wts[s];
    int ax = P->beam_axis, bx = (ax == 0) ? 1 : 0, cx = (ax == 2) ? 1 : 2;
    const int32_t *n = P->n;
    const double *dd = P->d;

    double u[6];
    or_block_uniforms(P->seed, h, P->stream, 0u, u);
    double zx, zy;
    or_box_muller(u[0], u[1], &zx, &zy);
    double eta = -log(u[2]);

    double E = P->spot_e[s];
    A->ledger[3] += E * w;

    double p[3], dir[3] = { 0.0, 0.0, 0.0 };
    p[bx] = P->spot_x[s] - P->origin[bx] - P->shift[bx] + P->spot_sigma[s] * zx;
    p[cx] = P->spot_y[s] - P->origin[cx] - P->shift[cx] + P->spot_sigma[s] * zy;
    p[ax] = P->beam_sign > 0 ? 0.0 : n[ax] * dd[ax];
    dir[ax] = (double)P->beam_sign;
    if (!(p[bx] >= 0.0 && p[bx] < n[bx] * dd[bx] &&
          p[cx] >= 0.0 && p[cx] < n[cx] * dd[cx])) {
        A->ledger[1] += E * w;                 /* never enters the grid */
        return;
    }
    int32_t iv[3];
    iv[bx] = (int32_t)floor(p[bx] / dd[bx]);
    iv[cx] = (int32_t)floor(p[cx] / dd[cx]);
    iv[ax] = P->beam_sign > 0 ? 0 : n[ax] - 1;

    double uthick = 0.0;                       /* radiation lengths so far */
    for (int64_t step = 0;; ++step) {
        if (step >= P->max_steps) {
            A->ledger[1] += E * w;
            A->status = OR_ESTEP;
            return;
        }
        A->steps += 1;
        size_t vox = ((size_t)iv[2] * n[1] + iv[1]) * n[0] + iv[0];
        int hu = P->hu[vox];
        double rho = or_rho(hu);
        double spr = or_spr(hu) * P->spr_scale;
        double R0 = or_range(E);
        double z_start = or_depth_of(P, p);
        if (R0 / spr <= OR_SMIN) {             /* residual range below s_min */
            A->edep[vox] += E * w;
            A->ledger[0] += E * w;
            or_depth_spread(P, A, z_start, z_start, E * w);
            A->end_depth[0] += w * z_start;
            A->end_depth[1] += w;
            A->end_depth[2] += w * z_start * z_start;
            return;
        }
        /* distance to the faces of the current voxel */
        double dbound = INFINITY;
        int across = -1;
        for (int k = 0; k < 3; ++k) {
            double t;
            if (dir[k] > 0.0) t = ((iv[k] + 1) * dd[k] - p[k]) / dir[k];
            else if (dir[k] < 0.0) t = (iv[k] * dd[k] - p[k]) / dir[k];
            else continue;
            if (t < 0.0) t = 0.0;
            if (t < dbound) { dbound = t; across = k; }
        }
        /* the step ends at the voxel boundary or after the physics length,
           whichever comes first */
        double s = fmax(OR_FSTEP * R0 / spr, OR_SMIN);
        int geom = 0;
        if (dbound <= s) { s = dbound; geom = 1; }

        double sw = s * spr;                   /* water-equivalent mm */
        double E1c, Emean;
        or_csda(E, R0, sw, &E1c, &Emean);
        int nuclear = 0;
        if (P->physics & OR_PHYS_NUC) {
            double sig = or_sigma_nuc(Emean);  /* 1/cm */
            double tau = sig * sw / 10.0;
            if (sig > 0.0 && tau >= eta) {
                nuclear = 1;
                sw = eta * 10.0 / sig;
                s = sw / spr;
                geom = 0;
                or_csda(E, R0, sw, &E1c, &Emean);
            } else {
                eta -= tau;
            }
        }
        or_block_uniforms(P->seed, h, P->stream, (uint32_t)(step + 1), u);
        double zA0, zA1, z1u, z2u, z1v, z2v;
        or_box_muller(u[0], u[1], &zA0, &zA1);
        or_box_muller(u[2], u[3], &z1u, &z2u);
        or_box_muller(u[4], u[5], &z1v, &z2v);

        double dE = E - E1c;
        if (P->physics & OR_PHYS_STRAG) {
            dE = or_straggle_loss(dE, or_bohr_var(E, sw), zA0);
            if (dE > E) dE = E;
        }
        double E1 = E - dE;

        if (nuclear) {
            double loc = OR_FLOC * E1;
            A->edep[vox] += (dE + loc) * w;
            A->ledger[0] += (dE + loc) * w;
            A->ledger[2] += (E1 - loc) * w;
            double zend = z_start + s * dir[ax] * P->beam_sign;
            or_depth_spread(P, A, z_start, zend, dE * w);
            or_depth_spread(P, A, zend, zend, loc * w);
            return;
        }
        if (E1 <= OR_ECUT) {
            A->edep[vox] += E * w;             /* dE + E1 */
            A->ledger[0] += E * w;
            double zend = z_start + s * dir[ax] * P->beam_sign;
            or_depth_spread(P, A, z_start, zend, dE * w);
            or_depth_spread(P, A, zend, zend, E1 * w);
            A->end_depth[0] += w * zend;
            A->end_depth[1] += w;
            A->end_depth[2] += w * zend * zend;
            return;
        }
        A->edep[vox] += dE * w;
        A->ledger[0] += dE * w;

        /* multiple Coulomb scattering over the step */
        double y1 = 0.0, y2 = 0.0, t1 = 0.0, t2 = 0.0;
        if (P->physics & OR_PHYS_MCS) {
            double du = s * rho / OR_X0_MM;
            double th2 = or_highland_theta2(Emean, uthick, du);
            uthick += du;
            double th0 = th2 > 0.0 ? sqrt(th2) : 0.0;
            or_mcs_plane(s, th0, z1u, z2u, &y1, &t1);
            or_mcs_plane(s, th0, z1v, z2v, &y2, &t2);
        }
        double e1[3], e2[3];
        or_frame(dir, e1, e2);
        double p0[3] = { p[0], p[1], p[2] };
        double dir0[3] = { dir[0], dir[1], dir[2] };
        for (int k = 0; k < 3; ++k) {
            p[k] = p[k] + s * dir[k] + y1 * e1[k] + y2 * e2[k];
            dir[k] = dir[k] + t1 * e1[k] + t2 * e2[k];
        }
        double nrm = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        for (int k = 0; k < 3; ++k) dir[k] /= nrm;
        E = E1;
        or_depth_spread(P, A, z_start, or_depth_of(P, p), dE * w);

        /* voxel update: the crossed axis advances by one and its coordinate
           is put on the crossed face; every other axis keeps its index while
           the position stays inside the voxel's closed extent [i d, (i+1) d]
           and takes floor(p/d) once the lateral displacement has carried it
           outside (keeping the index on a face avoids handing a particle
           that sits on an edge back and forth between two voxels)          */
        for (int k = 0; k < 3; ++k) {
            if (geom && k == across) {
                if (dir0[k] > 0.0) { iv[k] += 1; p[k] = iv[k] * dd[k]; }
                else { p[k] = iv[k] * dd[k]; iv[k] -= 1; }
            } else if (p[k] < iv[k] * dd[k] || p[k] > (iv[k] + 1) * dd[k]) {
                iv[k] = (int32_t)floor(p[k] / dd[k]);
            }
        }
        or_planes(P, A, p0, p, w);
        if (iv[0] < 0 || iv[0] >= n[0] || iv[1] < 0 || iv[1] >= n[1] ||
            iv[2] < 0 || iv[2] >= n[2]) {
            A->ledger[1] += E * w;
            return;
        }
    }
}

int or_transport(const or_run_params *P, or_run_out *O)
{
    or_init_tables();
    if (P->n_spots <= 0 || P->n_hist == 0 || P->hist_end > P->n_hist ||
        P->hist_begin > P->hist_end || P->beam_axis < 0 || P->beam_axis > 2 ||
        (P->beam_sign != 1 && P->beam_sign != -1))
        return OR_EINVAL;
    for (int64_t s = 0; s < P->n_spots; ++s)
        if (!(P->spot_e[s] >= 1.0 && P->spot_e[s] <= 250.0)) return OR_EINVAL;
    size_t nvox = (size_t)P->n[0] * P->n[1] * P->n[2];
    uint64_t *ns = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)P->n_spots);
    uint64_t *prefix = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(P->n_spots + 1));
    double *wts = (double *)malloc(sizeof(double) * (size_t)P->n_spots);
    if (!ns || !prefix || !wts) { free(ns); free(prefix); free(wts); return OR_ENOMEM; }
    int rc = or_allocate(P->n_spots, P->spot_protons, P->n_hist, ns);
    if (rc) { free(ns); free(prefix); free(wts); return rc; }
    double W = 0.0;
    for (int64_t s = 0; s < P->n_spots; ++s) W += (double)P->spot_protons[s];
    prefix[0] = 0;
    for (int64_t s = 0; s < P->n_spots; ++s) {
        prefix[s + 1] = prefix[s] + ns[s];
        /* history weight relative to the mean protons per history W/N */
        wts[s] = ns[s] ? (double)P->spot_protons[s] * (double)P->n_hist / ((double)ns[s] * W) : 0.0;
    }

    int nt = P->nthreads > 0 ? P->nthreads : 1;
    const uint64_t bc = P->batch_count > 1 ? P->batch_count : 1;
    const uint64_t bi = bc > 1 ? P->batch_index % bc : 0;
    const uint64_t first = P->hist_begin + (bi + bc - P->hist_begin % bc) % bc;
    const uint64_t count = first < P->hist_end ? (P->hist_end - first + bc - 1) / bc : 0;
    if ((uint64_t)nt > count && count > 0) nt = (int)count;
    if (nt < 1) nt = 1;
    or_acc *acc = (or_acc *)calloc((size_t)nt, sizeof(or_acc));
    int np = P->n_planes;
    int ok = acc != NULL;
    for (int t = 0; ok && t < nt; ++t) {
        acc[t].edep = (double *)calloc(nvox, sizeof(double));
        ok &= acc[t].edep != NULL;
        if (O->depth_dose) { acc[t].depth = (double *)calloc((size_t)P->n_depth_bins, sizeof(double)); ok &= acc[t].depth != NULL; }
        if (O->plane_w) {
            acc[t].pw = (double *)calloc((size_t)np, sizeof(double));
            acc[t].pm1 = (double *)calloc((size_t)(2 * np), sizeof(double));
            acc[t].pm2 = (double *)calloc((size_t)(2 * np), sizeof(double));
            ok &= acc[t].pw && acc[t].pm1 && acc[t].pm2;
        }
    }
    if (ok) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(static)
#endif
        for (int t = 0; t < nt; ++t) {
            uint64_t b = count * (uint64_t)t / (uint64_t)nt;
            uint64_t e = count * (uint64_t)(t + 1) / (uint64_t)nt;
            for (uint64_t k = b; k < e; ++k) or_history(P, prefix, wts, first + k * bc, &acc[t]);
        }
        /* fixed-order reduction */
        memset(O->ledger, 0, sizeof(O->ledger));
        O->end_depth[0] = O->end_depth[1] = O->end_depth[2] = 0.0;
        O->steps = 0;
        O->status = OR_OK;
        for (int t = 0; t < nt; ++t) {
            for (size_t i = 0; i < nvox; ++i) O->edep[i] += acc[t].edep[i];
            if (O->depth_dose)
                for (int k = 0; k < P->n_depth_bins; ++k) O->depth_dose[k] += acc[t].depth[k];
            if (O->plane_w)
                for (int k = 0; k < np; ++k) {
                    O->plane_w[k] += acc[t].pw[k];
                    O->plane_m1[k] += acc[t].pm1[k]; O->plane_m1[np + k] += acc[t].pm1[np + k];
                    O->plane_m2[k] += acc[t].pm2[k]; O->plane_m2[np + k] += acc[t].pm2[np + k];
                }
            for (int k = 0; k < 4; ++k) O->ledger[k] += acc[t].ledger[k];
            O->end_depth[0] += acc[t].end_depth[0];
            O->end_depth[1] += acc[t].end_depth[1];
            O->end_depth[2] += acc[t].end_depth[2];
            O->steps += acc[t].steps;
            if (acc[t].status) O->status = acc[t].status;
        }
        O->histories = count;
    }
    for (int t = 0; acc && t < nt; ++t) {
        free(acc[t].edep); free(acc[t].depth); free(acc[t].pw); free(acc[t].pm1); free(acc[t].pm2);
    }
    free(acc); free(ns); free(prefix); free(wts);
    return ok ? O->status : OR_ENOMEM;
}

/* One condensed-history step of a proton in an infinite uniform medium of
 * the given HU with energy E and cumulative radiation thickness u0, over a
 * step of s mm, drawn from the step-(step_index) uniforms of history h,
 * with the same pieces the transport uses.  Exposed so that the single-step
 * distributions (straggling variance, the correlated angle/displacement
 * moments) can be pinned.
 * out: [0] dE, [1] theta_1, [2] y_1, [3] theta_2, [4] y_2, [5] s (mm).     */
void or_single_step(int hu, double E, double u0, double s, uint64_t seed,
                    uint64_t h, uint32_t stream, uint32_t step_index,
                    double *out)
{
    or_init_tables();
    double rho = or_rho(hu), spr = or_spr(hu);
    double R0 = or_range(E);
    double sw = s * spr;
    double E1c, Emean;
    or_csda(E, R0, sw, &E1c, &Emean);
    double u[6];
    or_block_uniforms(seed, h, stream, step_index + 1, u);
    double zA0, zA1, z1u, z2u, z1v, z2v;
    or_box_muller(u[0], u[1], &zA0, &zA1);
    or_box_muller(u[2], u[3], &z1u, &z2u);
    or_box_muller(u[4], u[5], &z1v, &z2v);
    double dE = or_straggle_loss(E - E1c, or_bohr_var(E, sw), zA0);
    if (dE > E) dE = E;
    double th2 = or_highland_theta2(Emean, u0, s * rho / OR_X0_MM);
    double th0 = th2 > 0.0 ? sqrt(th2) : 0.0;
    out[0] = dE;
    or_mcs_plane(s, th0, z1u, z2u, &out[2], &out[1]);
    or_mcs_plane(s, th0, z1v, z2v, &out[4], &out[3]);
    out[5] = s;
}

/* theta0^2 and nuclear optical depth of one step of s mm from energy E in a
 * uniform medium, both taken at the step-mean energy as in the transport. */
double or_step_theta2(int hu, double E, double u0, double s)
{
    or_init_tables();
    double E1c, Emean;
    or_csda(E, or_range(E), s * or_spr(hu), &E1c, &Emean);
    return or_highland_theta2(Emean, u0, s * or_rho(hu) / OR_X0_MM);
}

double or_step_tau(int hu, double E, double s)
{
    or_init_tables();
    double sw = s * or_spr(hu);
    double E1c, Emean;
    or_csda(E, or_range(E), sw, &E1c, &Emean);
    return or_sigma_nuc(Emean) * sw / 10.0;
}

/* ======================================================================= */
/* Dose from deposited energy (Sec. 2.C: dose and density per CT voxel):   */
/*   D_i [Gy] = E_i [MeV] x W/N x 1.602176634e-13 J/MeV / (rho_i V_i 1e-3 kg) */
/* where E_i is the history-weighted deposit and W/N the mean protons per   */
/* history.                                                                 */
/* ======================================================================= */
void or_normalise(int64_t nvox, const double *edep, const double *rho,
                  double w_bar, double voxel_cm3, double *dose)
{
    for (int64_t i = 0; i < nvox; ++i)
        dose[i] = edep[i] * w_bar * OR_MEV_J / (rho[i] * voxel_cm3 * 1.0e-3);
}

/* ======================================================================= */
/* Delivery timeline (Sec. 2.B, App. A): integer-ns breathing and spot     */
/* clocks; each spot (or portion of a spot) is assigned to the breathing   */
/* phase during which it is delivered.                                     */
/*                                                                         */
/* Breathing clock of field f.  The clock starts (t = 0) at the beginning  */
/* of phase p0 of cycle 0; p0 is given or drawn as word 0 of Philox4x32-10 */
/* (counter (f, 0, 0, 0), key seed) mod N.  Cycle c lasts N t_c with       */
/* t_c = floor(T_c / N) (Sec. 2.B: t_ph ~ N(mu, sigma) / N, one draw per   */
/* cycle).  T_c = mu when sigma = 0; otherwise T_c = max(N, mu +           */
/* round(sigma Z_c)) with Z_c = sum of twelve uniforms - 6 (Irwin-Hall),   */
/* the uniforms being those of the blocks (f, c, 1, 0) and (f, c, 2, 0),  */
/* so that T_c = mu + floor((sigma (K - 6 (2^21 - 1)) + 2^20) / 2^21) with */
/* K the sum of their twelve 21-bit integers: exact integer arithmetic.    */
/*                                                                         */
/* Spill clock, common rules: spots of a field go in plan order; a layer   */
/* is a maximal run of equal layer ids; a spill of w protons lasts         */
/* floor(w 1e9 / rate) ns and is split over the phase slots it spans by    */
/* time share (floor for each portion, the remainder to the last).  Each   */
/* layer is painted `repaints` times (floor(p / R) per painting, the       */
/* remainder in the last) or, when max_protons_per_paint = m > 0, painted  */
/* until done with min(left, m) per spot and painting (isolayered          */
/* repainting with a maximum per spot delivery, Sec. 2.B).                 */
/*                                                                         */
/* synchrotron = 0 (the clock of Sec. 2.B): switch times precede every     */
/* spill but the first of a field (layer_switch_ns before a layer's first  */
/* spill, spot_switch_ns otherwise); gated delivery skips from a gate-off  */
/* phase to the start of the next gate_first phase and adds discard_ns.    */
/*                                                                         */
/* synchrotron = 1 (App. A): protons come in fills.  A fill starts with a  */
/* reset of layer_switch_ns (not for the field's first fill), then, when   */
/* gated, a hold until the gate is on, then the beam discard of            */
/* discard_ns, then extraction.  A new layer always takes a new fill.  A   */
/* fill holds fill_protons (0: unlimited) and extracts for at most         */
/* extraction_limit_ns after its extraction starts (0: unlimited).  Spills */
/* of one fill are separated by spot_switch_ns.  A spill that meets the    */
/* fill's charge, its time limit or a gate-off stops there: the part       */
/* delivered has the remaining charge, or floor(w elapsed / duration)      */
/* protons for a time cut, and the rest continues (without a spot switch) */
/* after the next extraction start: after a gate-off the beam holds until */
/* the gate is on and discards discard_ns again; after the charge or the  */
/* time limit a new fill starts.                                           */
/* ======================================================================= */
typedef struct {
    int32_t n_phases, start_phase, gated, gate_first, gate_last, repaints;
    int64_t period_ns, period_sigma_ns, spot_switch_ns, layer_switch_ns, discard_ns;
    uint64_t rate_protons_per_s, seed;
    int32_t synchrotron, reserved;
    uint64_t fill_protons;
    int64_t extraction_limit_ns;
    uint64_t max_protons_per_paint;
} or_delivery;

/* Irwin-Hall sum of the twelve 21-bit integers of blocks (a, b, c1, 0)
 * and (a, b, c1 + 1, 0) minus 6 (2^21 - 1): 2^21 times a standard deviate. */
static int64_t or_irwin_hall(uint64_t seed, uint32_t a, uint32_t b, uint32_t c1)
{
    int64_t K = 0;
    for (uint32_t blk = 0; blk < 2; ++blk) {
        uint32_t ctr[4] = { a, b, c1 + blk, 0u };
        uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
        uint32_t w[4];
        or_philox4x32_10(ctr, key, w);
        unsigned __int128 v = (unsigned __int128)w[0] | ((unsigned __int128)w[1] << 32) |
                              ((unsigned __int128)w[2] << 64) | ((unsigned __int128)w[3] << 96);
        for (int i = 0; i < 6; ++i) K += (int64_t)((v >> (21 * i)) & 0x1FFFFFu);
    }
    return K - 6 * (int64_t)0x1FFFFF;
}

/* mean + round(sigma Z) with Z = zk / 2^21 (round half up), exact. */
static int64_t or_gauss_ns(int64_t mean, int64_t sigma, int64_t zk)
{
    __int128 num = (__int128)sigma * zk + ((__int128)1 << 20);
    __int128 q = num >> 21;                    /* floor division by 2^21 */
    return mean + (int64_t)q;
}

typedef struct {
    const or_delivery *D;
    int32_t f;
    int64_t N;
    uint64_t cycle;
    int64_t cyc_start, tph;
} or_clock;

static int64_t or_cycle_tph(const or_clock *C, uint64_t c)
{
    int64_t T = C->D->period_ns;
    if (C->D->period_sigma_ns > 0) {
        T = or_gauss_ns(T, C->D->period_sigma_ns,
                        or_irwin_hall(C->D->seed, (uint32_t)C->f, (uint32_t)c, 1u));
        if (T < C->N) T = C->N;
    }
    return T / C->N;
}

static void or_clock_sync(or_clock *C, int64_t t)
{
    while (t >= C->cyc_start + C->N * C->tph) {
        C->cyc_start += C->N * C->tph;
        C->cycle += 1;
        C->tph = or_cycle_tph(C, C->cycle);
    }
}

static uint32_t or_phase_at(or_clock *C, int64_t t)
{
    or_clock_sync(C, t);
    return (uint32_t)((t - C->cyc_start) / C->tph);
}

static int64_t or_slot_end(or_clock *C, int64_t t)
{
    or_clock_sync(C, t);
    return C->cyc_start + ((t - C->cyc_start) / C->tph + 1) * C->tph;
}

static int or_gate_on(const or_clock *C, uint32_t ph)
{
    return !C->D->gated || ((int32_t)ph >= C->D->gate_first && (int32_t)ph <= C->D->gate_last);
}

/* the start of the next gate-on slot at or after t */
static int64_t or_hold(or_clock *C, int64_t t)
{
    while (!or_gate_on(C, or_phase_at(C, t))) t = or_slot_end(C, t);
    return t;
}

/* the end of the gate-on run containing t (looked up on a copy of the clock) */
static int64_t or_gate_off_after(const or_clock *C, int64_t t)
{
    or_clock L = *C;
    while (or_gate_on(&L, or_phase_at(&L, t))) t = or_slot_end(&L, t);
    return t;
}

/* Deliver w protons over [t, end), split at slot ends by time share. */
static void or_deposit(or_clock *C, int64_t t, int64_t end, uint64_t w, uint64_t *pp,
                       int64_t n_spots, int64_t q)
{
    if (w == 0) return;
    if (end <= t) {
        pp[(size_t)or_phase_at(C, t) * (size_t)n_spots + (size_t)q] += w;
        return;
    }
    const uint64_t dur = (uint64_t)(end - t);
    uint64_t given = 0;
    while (t < end) {
        int64_t se = or_slot_end(C, t);
        int64_t e = se < end ? se : end;
        uint32_t ph = or_phase_at(C, t);
        uint64_t pj = (e == end) ? w - given
                                 : (uint64_t)((unsigned __int128)w * (uint64_t)(e - t) / dur);
        given += pj;
        pp[(size_t)ph * (size_t)n_spots + (size_t)q] += pj;
        t = e;
    }
}

static int64_t or_spill_ns(uint64_t w, uint64_t rate)
{
    return (int64_t)((unsigned __int128)w * 1000000000u / rate);
}

/* Parameters that make every fill and every gate window deliver at least
 * one proton (so the clock always advances): checked on both sides.     */
static int or_delivery_ok(const or_delivery *D)
{
    if (D->n_phases <= 0 || D->repaints <= 0 || D->period_ns <= 0 || D->rate_protons_per_s == 0 ||
        D->period_sigma_ns < 0 || D->spot_switch_ns < 0 || D->layer_switch_ns < 0 ||
        D->discard_ns < 0 || D->start_phase >= D->n_phases || D->extraction_limit_ns < 0)
        return 0;
    if (D->max_protons_per_paint > 0 && D->repaints != 1) return 0;
    if (D->synchrotron != 0 && D->synchrotron != 1) return 0;
    /* shortest cycle: mu - 6 sigma (the Irwin-Hall bound), at least N ns */
    __int128 tmin = (__int128)D->period_ns - 6 * (__int128)D->period_sigma_ns;
    if (tmin < D->n_phases) return 0;
    int64_t tph_min = (int64_t)(tmin / D->n_phases);
    int64_t proton_ns = (int64_t)((1000000000ull + D->rate_protons_per_s - 1) / D->rate_protons_per_s);
    if (D->gated) {
        if (D->gate_first < 0 || D->gate_last >= D->n_phases || D->gate_first > D->gate_last) return 0;
        int64_t window = (int64_t)(D->gate_last - D->gate_first + 1) * tph_min;
        if (D->discard_ns >= window) return 0;
        if (D->synchrotron && window - D->discard_ns < proton_ns) return 0;
    }
    if (D->synchrotron && D->extraction_limit_ns > 0 && D->extraction_limit_ns < proton_ns) return 0;
    return 1;
}

typedef struct {                          /* synchrotron fill state */
    int in_fill, fills, spills, empty;
    int64_t ext_start;
    uint64_t left, got;
} or_fill;

#define OR_MAX_EMPTY_FILLS 64

/* Start a fill's extraction (App. A): reset, hold for the gate, discard.
 * Returns -1 when too many fills in a row delivered nothing.            */
static int64_t or_fill_start(or_clock *C, or_fill *F, int64_t t)
{
    const or_delivery *D = C->D;
    if (F->fills > 0) {
        F->empty = F->got ? 0 : F->empty + 1;
        if (F->empty > OR_MAX_EMPTY_FILLS) return -1;
        t += D->layer_switch_ns;
    }
    F->fills += 1;
    if (D->gated) t = or_hold(C, t);
    t += D->discard_ns;
    F->ext_start = t;
    F->left = D->fill_protons;
    F->in_fill = 1;
    F->spills = 0;
    F->got = 0;
    return t;
}

/* One spot portion of w protons under the synchrotron rules; -1 when the
 * delivery makes no progress.                                           */
static int64_t or_sync_spill(or_clock *C, or_fill *F, int64_t t, uint64_t w, uint64_t *pp,
                             int64_t n_spots, int64_t q)
{
    const or_delivery *D = C->D;
    int first = 1;
    while (w > 0) {
        if (!F->in_fill) {
            if ((t = or_fill_start(C, F, t)) < 0) return -1;
        } else if (first && F->spills > 0) {
            t += D->spot_switch_ns;
        }
        first = 0;
        const int64_t lim = D->extraction_limit_ns > 0 ? F->ext_start + D->extraction_limit_ns : INT64_MAX;
        if (D->gated && !or_gate_on(C, or_phase_at(C, t))) {
            const int64_t resume = or_hold(C, t) + D->discard_ns;   /* paused at a gate-off */
            if (resume >= lim) {                 /* the fill expires while held */
                if (t < lim) t = lim;
                F->in_fill = 0;
                continue;
            }
            t = resume;
        }
        if (t >= lim) { F->in_fill = 0; continue; }
        uint64_t part = w;
        if (D->fill_protons > 0 && F->left < part) part = F->left;
        const int64_t dur = or_spill_ns(part, D->rate_protons_per_s);
        int64_t end = t + dur;
        int cut = 0;                                    /* 1: time limit, 2: gate-off */
        if (end > lim) { end = lim; cut = 1; }
        if (D->gated) {
            int64_t off = or_gate_off_after(C, t);
            if (end > off) { end = off; cut = 2; }
        }
        uint64_t now = part;
        if (cut) now = (uint64_t)((unsigned __int128)part * (uint64_t)(end - t) / (uint64_t)dur);
        or_deposit(C, t, end, now, pp, n_spots, q);
        t = end;
        w -= now;
        F->got += now;
        F->spills += 1;
        if (D->fill_protons > 0) F->left -= now;
        if (cut == 1 || (D->fill_protons > 0 && F->left == 0)) F->in_fill = 0;
    }
    return t;
}

/* Simple-clock gate: from a gate-off phase, skip to the start of the next
 * gate_first phase and add the beam discard.                            */
static int64_t or_wait_gate(or_clock *C, int64_t t)
{
    if (C->D->gated && !or_gate_on(C, or_phase_at(C, t))) t = or_hold(C, t) + C->D->discard_ns;
    return t;
}

int or_timeline(int64_t n_spots, const uint64_t *protons, const int32_t *layer,
                const int32_t *field, const or_delivery *D, uint64_t *pp,
                int64_t *field_end_ns, int32_t *start_phase_out, int32_t n_fields)
{
    if (n_spots <= 0 || n_fields <= 0 || !or_delivery_ok(D)) return OR_EINVAL;
    for (int64_t s = 0; s < n_spots; ++s)
        if (field[s] < 0 || field[s] >= n_fields) return OR_EINVAL;
    memset(pp, 0, sizeof(uint64_t) * (size_t)(n_spots * D->n_phases));
    uint64_t *left = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n_spots);
    if (!left) return OR_ENOMEM;
    const uint64_t R = (uint64_t)D->repaints, cap = D->max_protons_per_paint;
    int rc = OR_OK;
    for (int32_t f = 0; f < n_fields && rc == OR_OK; ++f) {
        uint32_t p0;
        if (D->start_phase >= 0) {
            p0 = (uint32_t)D->start_phase;
        } else {
            /* random start phase: word 0 of Philox(counter (f,0,0,0), key seed) mod N */
            uint32_t ctr[4] = { (uint32_t)f, 0u, 0u, 0u };
            uint32_t key[2] = { (uint32_t)D->seed, (uint32_t)(D->seed >> 32) };
            uint32_t w[4];
            or_philox4x32_10(ctr, key, w);
            p0 = w[0] % (uint32_t)D->n_phases;
        }
        start_phase_out[f] = (int32_t)p0;
        or_clock C = { D, f, D->n_phases, 0u, 0, 0 };
        C.tph = or_cycle_tph(&C, 0);
        C.cyc_start = -(int64_t)p0 * C.tph;
        or_fill F = { 0, 0, 0, 0, 0, 0, 0 };
        int64_t t = 0;
        int delivered_any = 0;
        int64_t s = 0;
        while (s < n_spots && rc == OR_OK) {
            if (field[s] != f) { ++s; continue; }
            int64_t l0 = s, l1 = s;
            for (int64_t k = s + 1; k < n_spots; ++k) {
                if (field[k] != f) continue;
                if (layer[k] != layer[l0]) break;
                l1 = k;
            }
            s = l1 + 1;
            int layer_started = 0;
            F.in_fill = 0;                          /* a new energy takes a new fill */
            for (int64_t q = l0; q <= l1; ++q) left[q] = protons[q];
            for (uint64_t r = 0; rc == OR_OK; ++r) {
                if (cap == 0 && r == R) break;
                int any = 0;
                for (int64_t q = l0; q <= l1; ++q) {
                    if (field[q] != f) continue;
                    uint64_t w;
                    if (cap > 0) {
                        w = left[q] < cap ? left[q] : cap;
                    } else {
                        w = protons[q] / R;
                        if (r == R - 1) w += protons[q] % R;
                    }
                    if (w == 0) continue;
                    left[q] -= w;
                    any = 1;
                    if (D->synchrotron) {
                        t = or_sync_spill(&C, &F, t, w, pp, n_spots, q);
                        if (t < 0) { rc = OR_ESTEP; break; }
                        continue;
                    }
                    if (delivered_any)
                        t += layer_started ? D->spot_switch_ns : D->layer_switch_ns;
                    delivered_any = 1;
                    layer_started = 1;
                    /* spill time of this portion, ns */
                    const int64_t dur = or_spill_ns(w, D->rate_protons_per_s);
                    t = or_wait_gate(&C, t);
                    if (dur == 0) {
                        pp[(size_t)or_phase_at(&C, t) * (size_t)n_spots + (size_t)q] += w;
                        continue;
                    }
                    /* split over slots by time share, pausing at gate-offs */
                    int64_t rem = dur;
                    uint64_t given = 0;
                    while (rem > 0) {
                        t = or_wait_gate(&C, t);
                        int64_t seg = or_slot_end(&C, t) - t;
                        int64_t d = rem < seg ? rem : seg;
                        uint32_t ph = or_phase_at(&C, t);
                        t += d;
                        rem -= d;
                        uint64_t pj = rem > 0 ? (uint64_t)((unsigned __int128)w * (uint64_t)d / (uint64_t)dur)
                                              : w - given;
                        given += pj;
                        pp[(size_t)ph * (size_t)n_spots + (size_t)q] += pj;
                    }
                }
                if (cap > 0 && !any) break;
            }
        }
        field_end_ns[f] = t;
    }
    free(left);
    return rc;
}

/* ======================================================================= */
/* Uncertainty trials (Sec. 2.B, the 25-trial study): trial k's delivery   */
/* draws, from Philox4x32-10 under key `seed`, a breathing period from the */
/* discrete uniform set {min, min + step, ..., max} (word 0 of block (k,   */
/* 0, 3, 0) mod the set size) and each synchrotron parameter from          */
/* N(mean, sigma) (Irwin-Hall blocks (k, j, 4, 0), (k, j, 5, 0) for        */
/* parameter j = 0 spot switch, 1 layer switch, 2 discard, 3 rate, 4 fill  */
/* charge, 5 extraction limit; round half up; clamped at 0, the rate at   */
/* 1).  The trial's own seed, which draws its start phase and breathing    */
/* cycles, is seed + k 0x9E3779B97F4A7C15 (mod 2^64).                      */
/* ======================================================================= */
typedef struct {
    int64_t period_min_ns, period_max_ns, period_step_ns;
    int64_t spot_switch_sigma_ns, layer_switch_sigma_ns, discard_sigma_ns;
    int64_t rate_sigma, fill_protons_sigma, extraction_limit_sigma_ns;
} or_spread;

static int64_t or_clamp0(int64_t v) { return v < 0 ? 0 : v; }

int or_trial_delivery(const or_delivery *mean, const or_spread *S, uint64_t trial, or_delivery *out)
{
    *out = *mean;
    const uint64_t seed = mean->seed;
    if (S->period_max_ns > S->period_min_ns) {
        if (S->period_step_ns <= 0 || S->period_min_ns <= 0) return OR_EINVAL;
        uint64_t n = (uint64_t)((S->period_max_ns - S->period_min_ns) / S->period_step_ns) + 1;
        uint32_t ctr[4] = { (uint32_t)trial, 0u, 3u, 0u };
        uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
        uint32_t w[4];
        or_philox4x32_10(ctr, key, w);
        out->period_ns = S->period_min_ns + (int64_t)(w[0] % n) * S->period_step_ns;
    }
    const int64_t sig[6] = { S->spot_switch_sigma_ns, S->layer_switch_sigma_ns, S->discard_sigma_ns,
                             S->rate_sigma, S->fill_protons_sigma, S->extraction_limit_sigma_ns };
    int64_t val[6] = { mean->spot_switch_ns, mean->layer_switch_ns, mean->discard_ns,
                       (int64_t)mean->rate_protons_per_s, (int64_t)mean->fill_protons,
                       mean->extraction_limit_ns };
    for (int j = 0; j < 6; ++j) {
        if (sig[j] < 0) return OR_EINVAL;
        if (sig[j] == 0) continue;
        val[j] = or_clamp0(or_gauss_ns(val[j], sig[j], or_irwin_hall(seed, (uint32_t)trial, (uint32_t)j, 4u)));
    }
    out->spot_switch_ns = val[0];
    out->layer_switch_ns = val[1];
    out->discard_ns = val[2];
    out->rate_protons_per_s = (uint64_t)(val[3] < 1 ? 1 : val[3]);
    out->fill_protons = (uint64_t)val[4];
    out->extraction_limit_ns = val[5];
    out->seed = seed + trial * 0x9E3779B97F4A7C15ull;
    return OR_OK;
}

/* 2^21 Z of cycle c of field f (exposed for the distribution pins). */
int64_t or_breathing_deviate(uint64_t seed, int32_t f, uint64_t c)
{
    return or_irwin_hall(seed, (uint32_t)f, (uint32_t)c, 1u);
}

/* A component of a field given at voxel centres (x fastest), interpolated
 * trilinearly at q in voxel-centre index space (voxel i's centre at i),
 * clamped to the edge values outside the outermost centres.  FP64.        */
static double or_d_sample(const float *comp, const int32_t *n, const double q[3])
{
    int32_t lo[3], hi[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(q[a]);
        f[a] = q[a] - fl;
        int32_t k = (int32_t)fl;
        lo[a] = k < 0 ? 0 : (k > n[a] - 1 ? n[a] - 1 : k);
        hi[a] = k + 1 < 0 ? 0 : (k + 1 > n[a] - 1 ? n[a] - 1 : k + 1);
    }
    double v = 0.0;
    for (int c = 0; c < 8; ++c) {
        int32_t x = (c & 1) ? hi[0] : lo[0];
        int32_t y = (c & 2) ? hi[1] : lo[1];
        int32_t z = (c & 4) ? hi[2] : lo[2];
        double w = ((c & 1) ? f[0] : 1.0 - f[0]) * ((c & 2) ? f[1] : 1.0 - f[1]) *
                   ((c & 4) ? f[2] : 1.0 - f[2]);
        v += w * (double)comp[((size_t)z * n[1] + y) * n[0] + x];
    }
    return v;
}

/* ======================================================================= */
/* Energy/mass-transfer accumulation (Sec. 2.D.2, Eqs. 4-6) and the phase  */
/* sum of Eq. 2, in FP64.                                                  */
/*                                                                         */
/* Each voxel j of every source phase S != R is split into nsub[0] x       */
/* nsub[1] x nsub[2] subvoxels; the centre of subvoxel k, in voxel-centre  */
/* index space q = j + (k + 1/2)/nsub - 1/2, is moved by the DVF of S      */
/* (trilinear between voxel centres, edge-clamped: or_d_sample), giving    */
/* the cell coordinate t = q + 1/2 + u / d, and lands in the reference     */
/* voxel i = floor(t) whose half-open cell [i, i + 1) holds it.  Subvoxel  */
/* mass is M = rho_j v_k and energy E = M D_j (Eq. 4); D_i^S = sum E / sum */
/* M over the subvoxels landing in i (Eqs. 5, 6), 0 where none lands; D_i  */
/* = D_i^R + sum_S D_i^S (Eq. 2), zero outside the mask.  Points landing   */
/* outside the grid are dropped and counted.                               */
/*                                                                         */
/* Ties.  The target voxel is an integer decided by floating point: a      */
/* point within eps (cell units) of a cell face may be decided either way  */
/* by any finite-precision implementation.  Besides its own decision, the  */
/* oracle reports such points as ambiguous and bounds what any decision    */
/* of them can give: with the unambiguous points fixed, the D_i^S that     */
/* results when the ambiguous ones go to any of their candidate cells is a */
/* mass-weighted mean of the unambiguous ratio and the source doses D_j of */
/* the candidates (or 0 when nothing lands), so it lies in [lo_i^S,        */
/* hi_i^S], the range of those values; lo_i and hi_i sum these bounds over */
/* the phases like Eq. 2.  Without ambiguous points lo = hi = accum.       */
/* counts: [0] dropped (this decision), [1] dropped under every decision   */
/* of the ambiguous points, [2] dropped under some decision, [3] ambiguous */
/* subvoxels.                                                              */
/* ======================================================================= */
static int or_cell_candidates(const double t[3], const int32_t n[3], double eps,
                              int32_t cand[8][3], int *n_out)
{
    int32_t lo[3], alt[3];
    int amb = 0;
    for (int a = 0; a < 3; ++a) {
        lo[a] = (int32_t)floor(t[a]);
        double face = floor(t[a] + 0.5);              /* nearest cell face */
        alt[a] = lo[a];
        if (fabs(t[a] - face) < eps) {
            alt[a] = (lo[a] == (int32_t)face) ? lo[a] - 1 : (int32_t)face;
            amb = 1;
        }
    }
    int m = 0, out = 0;
    for (int c = 0; c < 8; ++c) {
        int32_t v[3];
        int skip = 0;
        for (int a = 0; a < 3; ++a) {
            if (c & (1 << a)) { if (alt[a] == lo[a]) { skip = 1; break; } v[a] = alt[a]; }
            else v[a] = lo[a];
        }
        if (skip) continue;
        cand[m][0] = v[0]; cand[m][1] = v[1]; cand[m][2] = v[2];
        if (v[0] < 0 || v[0] >= n[0] || v[1] < 0 || v[1] >= n[1] || v[2] < 0 || v[2] >= n[2]) ++out;
        ++m;
    }
    *n_out = m;
    return amb ? (out == m ? 2 : (out ? 1 : 0)) + 4 : (out ? 2 : 0);
}

int or_emtm(const int32_t n[3], const float dmm[3], int32_t n_phases,
            int32_t ref_phase, const int32_t nsub[3], const float *dose,
            const float *rho, const float *dvf, const uint8_t *mask, double eps,
            double *accum, double *e_sum, double *m_sum, double *accum_lo,
            double *accum_hi, uint64_t counts[4])
{
    if (n_phases <= 0 || ref_phase < 0 || ref_phase >= n_phases ||
        nsub[0] <= 0 || nsub[1] <= 0 || nsub[2] <= 0)
        return OR_EINVAL;
    size_t nvox = (size_t)n[0] * n[1] * n[2];
    double *E = (double *)calloc(nvox, sizeof(double));
    double *M = (double *)calloc(nvox, sizeof(double));
    double *E0 = (double *)calloc(nvox, sizeof(double));
    double *M0 = (double *)calloc(nvox, sizeof(double));
    double *clo = (double *)malloc(nvox * sizeof(double));
    double *chi = (double *)malloc(nvox * sizeof(double));
    if (!E || !M || !E0 || !M0 || !clo || !chi) {
        free(E); free(M); free(E0); free(M0); free(clo); free(chi);
        return OR_ENOMEM;
    }
    for (size_t i = 0; i < nvox; ++i) {
        double r = (double)dose[(size_t)ref_phase * nvox + i];
        accum[i] = r;
        if (accum_lo) accum_lo[i] = r;
        if (accum_hi) accum_hi[i] = r;
    }
    uint64_t cnt[4] = { 0, 0, 0, 0 };
    for (int32_t S = 0; S < n_phases; ++S) {
        if (S == ref_phase) continue;
        memset(E, 0, nvox * sizeof(double));
        memset(M, 0, nvox * sizeof(double));
        memset(E0, 0, nvox * sizeof(double));
        memset(M0, 0, nvox * sizeof(double));
        for (size_t i = 0; i < nvox; ++i) { clo[i] = INFINITY; chi[i] = -INFINITY; }
        const float *ds = dose + (size_t)S * nvox;
        const float *rs = rho + (size_t)S * nvox;
        for (int32_t jz = 0; jz < n[2]; ++jz)
        for (int32_t jy = 0; jy < n[1]; ++jy)
        for (int32_t jx = 0; jx < n[0]; ++jx) {
            size_t j = ((size_t)jz * n[1] + jy) * n[0] + jx;
            double m = (double)rs[j];
            double dj = (double)ds[j];
            double e = m * dj;
            int32_t jj[3] = { jx, jy, jz };
            for (int32_t kz = 0; kz < nsub[2]; ++kz)
            for (int32_t ky = 0; ky < nsub[1]; ++ky)
            for (int32_t kx = 0; kx < nsub[0]; ++kx) {
                int32_t kk[3] = { kx, ky, kz };
                double q[3], t[3];
                for (int a = 0; a < 3; ++a)
                    q[a] = (double)jj[a] + ((double)kk[a] + 0.5) / (double)nsub[a] - 0.5;
                for (int a = 0; a < 3; ++a) {
                    double u = dvf ? or_d_sample(dvf + ((size_t)S * 3 + a) * nvox, n, q) : 0.0;
                    t[a] = q[a] + 0.5 + u / (double)dmm[a];
                }
                int32_t ix = (int32_t)floor(t[0]), iy = (int32_t)floor(t[1]), iz = (int32_t)floor(t[2]);
                int inside = !(ix < 0 || ix >= n[0] || iy < 0 || iy >= n[1] || iz < 0 || iz >= n[2]);
                size_t i = inside ? ((size_t)iz * n[1] + iy) * n[0] + ix : 0;
                if (inside) { E[i] += e; M[i] += m; } else ++cnt[0];
                int32_t cand[8][3];
                int nc = 0;
                int cls = or_cell_candidates(t, n, eps, cand, &nc);
                if (!(cls & 4)) {                       /* unambiguous */
                    if (inside) { E0[i] += e; M0[i] += m; }
                    else { ++cnt[1]; ++cnt[2]; }
                    continue;
                }
                ++cnt[3];
                if ((cls & 3) == 2) ++cnt[1];          /* every candidate outside */
                if (cls & 3) ++cnt[2];                 /* some candidate outside */
                if (!(m > 0.0)) continue;              /* carries no mass */
                for (int c = 0; c < nc; ++c) {
                    if (cand[c][0] < 0 || cand[c][0] >= n[0] || cand[c][1] < 0 ||
                        cand[c][1] >= n[1] || cand[c][2] < 0 || cand[c][2] >= n[2])
                        continue;
                    size_t ic = ((size_t)cand[c][2] * n[1] + cand[c][1]) * n[0] + cand[c][0];
                    if (dj < clo[ic]) clo[ic] = dj;
                    if (dj > chi[ic]) chi[ic] = dj;
                }
            }
        }
        for (size_t i = 0; i < nvox; ++i) {
            if (M[i] > 0.0) accum[i] += E[i] / M[i];
            if (e_sum) e_sum[i] += E[i];
            if (m_sum) m_sum[i] += M[i];
            double base = M0[i] > 0.0 ? E0[i] / M0[i] : 0.0;
            double lo = base, hi = base;
            if (clo[i] <= chi[i]) {                    /* an ambiguous point may land here */
                if (clo[i] < lo) lo = clo[i];
                if (chi[i] > hi) hi = chi[i];
            }
            if (accum_lo) accum_lo[i] += lo;
            if (accum_hi) accum_hi[i] += hi;
        }
    }
    if (mask)
        for (size_t i = 0; i < nvox; ++i)
            if (!mask[i]) {
                accum[i] = 0.0;
                if (accum_lo) accum_lo[i] = 0.0;
                if (accum_hi) accum_hi[i] = 0.0;
            }
    if (counts) for (int k = 0; k < 4; ++k) counts[k] = cnt[k];
    free(E); free(M); free(E0); free(M0); free(clo); free(chi);
    return OR_OK;
}

/* ======================================================================= */
/* Dose-interpolation accumulation (Sec. 2.D.2, Eq. 3) and the phase sum of */
/* Eq. 2.                                                                   */
/*                                                                          */
/* For every source phase S != R and every reference voxel i, the voxel is  */
/* split into nsub[0] x nsub[1] x nsub[2] subvoxels; the centre r_ik of     */
/* each is carried to phase S by the reference-to-source field T^{R->S}     */
/* (its displacement, in mm, given at the reference voxel centres and       */
/* interpolated trilinearly between them), the dose of S is interpolated    */
/* trilinearly at the carried point, and D_i^S is the mean over the         */
/* subvoxels (Eq. 3).  D_i = D_i^R + sum_S D_i^S (Eq. 2), zero outside the  */
/* mask.  Both interpolations use the values at voxel centres and clamp to  */
/* the edge outside them (a point carried past the grid takes the dose of   */
/* the nearest edge voxel).  Everything is FP64.                            */
/* ======================================================================= */
int or_dim(const int32_t n[3], const float dmm[3], int32_t n_phases, int32_t ref_phase,
           const int32_t nsub[3], const float *dose, const float *dvf, const uint8_t *mask,
           double *accum)
{
    if (n_phases <= 0 || ref_phase < 0 || ref_phase >= n_phases ||
        nsub[0] <= 0 || nsub[1] <= 0 || nsub[2] <= 0)
        return OR_EINVAL;
    size_t nvox = (size_t)n[0] * n[1] * n[2];
    const double nk = (double)nsub[0] * nsub[1] * nsub[2];
    for (size_t i = 0; i < nvox; ++i) accum[i] = (double)dose[(size_t)ref_phase * nvox + i];
    for (int32_t S = 0; S < n_phases; ++S) {
        if (S == ref_phase) continue;
        const float *ds = dose + (size_t)S * nvox;
        for (int32_t iz = 0; iz < n[2]; ++iz)
        for (int32_t iy = 0; iy < n[1]; ++iy)
        for (int32_t ix = 0; ix < n[0]; ++ix) {
            int32_t ii[3] = { ix, iy, iz };
            double sum = 0.0;
            for (int32_t kz = 0; kz < nsub[2]; ++kz)
            for (int32_t ky = 0; ky < nsub[1]; ++ky)
            for (int32_t kx = 0; kx < nsub[0]; ++kx) {
                int32_t kk[3] = { kx, ky, kz };
                /* r_ik in voxel-centre index space (voxel i's centre at i) */
                double q[3], t[3];
                for (int a = 0; a < 3; ++a)
                    q[a] = (double)ii[a] + ((double)kk[a] + 0.5) / (double)nsub[a] - 0.5;
                /* T^{R->S}(r_ik) = r_ik + displacement, mm -> voxels */
                for (int a = 0; a < 3; ++a) {
                    double disp = dvf ? or_d_sample(dvf + ((size_t)S * 3 + a) * nvox, n, q) : 0.0;
                    t[a] = q[a] + disp / (double)dmm[a];
                }
                sum += or_d_sample(ds, n, t);
            }
            accum[((size_t)iz * n[1] + iy) * n[0] + ix] += sum / nk;
        }
    }
    if (mask)
        for (size_t i = 0; i < nvox; ++i) if (!mask[i]) accum[i] = 0.0;
    return OR_OK;
}

/* ======================================================================= */
/* Decoding a registration's vector grid (App. B, Eqs. 7-8) onto the CT     */
/* grid, in FP64.                                                           */
/*                                                                          */
/* Grid voxel (i, j, k) sits at r0 = start + i dX U + j dY V + k dZ W with  */
/* W = U x V (Eq. 8) and maps to r_f = M_post (M_pre r0 + Delta_ijk)        */
/* (Eq. 7).  A point between grid voxels maps to the trilinear interpolant  */
/* of the r_f of the eight around it.  For each CT voxel centre p (patient  */
/* frame: origin + (idx + 1/2) d) the continuous grid index is              */
/* (U.(p - start)/dX, V.(p - start)/dY, W.(p - start)/dZ); the voxel is     */
/* inside when every component lies in [0, N - 1], and then its             */
/* displacement is r_f(p) - p; outside, the displacement is 0 and the       */
/* voxel is left out of the mask (Sec. 2.D.2: dose is reported only where   */
/* every DVF is defined).                                                   */
/*                                                                          */
/* Inside-ness is an integer decided by floating point: a voxel whose       */
/* continuous index lies within eps (grid-index units) of 0 or N - 1 on     */
/* some axis, and clearly inside on the others, may be decided either way  */
/* by a finite-precision implementation, and is flagged in `ambiguous` (the */
/* oracle's own decision is the FP64 one above).  pre, post: row-major      */
/* 4 x 4.  delta: (Dx, Dy, Dz) per grid voxel, x fastest.                   */
/* ======================================================================= */
static void or_affine(const float *M, const double v[3], double out[3])
{
    for (int r = 0; r < 3; ++r)
        out[r] = (double)M[4 * r + 0] * v[0] + (double)M[4 * r + 1] * v[1] +
                 (double)M[4 * r + 2] * v[2] + (double)M[4 * r + 3];
}

int or_dvf_decode(const int32_t gn[3], const float gstart[3], const float gsp[3],
                  const float U[3], const float V[3], const float pre[16],
                  const float post[16], const float *delta, const int32_t n[3],
                  const float d[3], const float origin[3], double eps, double *disp,
                  uint8_t *inside, uint8_t *ambiguous)
{
    if (gn[0] <= 0 || gn[1] <= 0 || gn[2] <= 0 || !(gsp[0] > 0) || !(gsp[1] > 0) ||
        !(gsp[2] > 0))
        return OR_EINVAL;
    const size_t ng = (size_t)gn[0] * gn[1] * gn[2];
    const size_t nvox = (size_t)n[0] * n[1] * n[2];
    double *rf = (double *)malloc(3 * ng * sizeof(double));
    if (!rf) return OR_ENOMEM;
    const double Ud[3] = { U[0], U[1], U[2] }, Vd[3] = { V[0], V[1], V[2] };
    const double Wd[3] = { Ud[1] * Vd[2] - Ud[2] * Vd[1],     /* W = U x V */
                           Ud[2] * Vd[0] - Ud[0] * Vd[2],
                           Ud[0] * Vd[1] - Ud[1] * Vd[0] };
    for (int32_t k = 0; k < gn[2]; ++k)
    for (int32_t j = 0; j < gn[1]; ++j)
    for (int32_t i = 0; i < gn[0]; ++i) {
        size_t g = ((size_t)k * gn[1] + j) * gn[0] + i;
        double r0[3], a[3], b[3];
        for (int c = 0; c < 3; ++c)           /* Eq. 8 */
            r0[c] = (double)gstart[c] + (double)i * gsp[0] * Ud[c] + (double)j * gsp[1] * Vd[c] +
                    (double)k * gsp[2] * Wd[c];
        or_affine(pre, r0, a);                /* Eq. 7 */
        for (int c = 0; c < 3; ++c) a[c] += (double)delta[3 * g + c];
        or_affine(post, a, b);
        for (int c = 0; c < 3; ++c) rf[c * ng + g] = b[c];
    }
    const double *axes[3] = { Ud, Vd, Wd };
    for (int32_t iz = 0; iz < n[2]; ++iz)
    for (int32_t iy = 0; iy < n[1]; ++iy)
    for (int32_t ix = 0; ix < n[0]; ++ix) {
        size_t v = ((size_t)iz * n[1] + iy) * n[0] + ix;
        int32_t ii[3] = { ix, iy, iz };
        double p[3], rel[3];
        for (int c = 0; c < 3; ++c) {
            p[c] = (double)origin[c] + ((double)ii[c] + 0.5) * (double)d[c];
            rel[c] = p[c] - (double)gstart[c];
        }
        double q[3];
        int in = 1, near = 0, far_out = 0;
        for (int a = 0; a < 3; ++a) {
            const double *ax = axes[a];
            q[a] = (ax[0] * rel[0] + ax[1] * rel[1] + ax[2] * rel[2]) / (double)gsp[a];
            if (!(q[a] >= 0.0 && q[a] <= (double)(gn[a] - 1))) in = 0;
            if (fabs(q[a]) < eps || fabs(q[a] - (double)(gn[a] - 1)) < eps) near = 1;
            else if (!(q[a] > 0.0 && q[a] < (double)(gn[a] - 1))) far_out = 1;
        }
        /* a decision can change only near a face and not outside on another axis */
        int amb = near && !far_out;
        inside[v] = (uint8_t)in;
        if (ambiguous) ambiguous[v] = (uint8_t)amb;
        if (!in) {
            for (int c = 0; c < 3; ++c) disp[c * nvox + v] = 0.0;
            continue;
        }
        int32_t lo[3], hi[3];
        double f[3];
        for (int a = 0; a < 3; ++a) {
            double fl = floor(q[a]);
            f[a] = q[a] - fl;
            lo[a] = (int32_t)fl;
            hi[a] = lo[a] + 1 > gn[a] - 1 ? gn[a] - 1 : lo[a] + 1;
        }
        for (int c = 0; c < 3; ++c) {
            double val = 0.0;
            for (int corner = 0; corner < 8; ++corner) {
                int32_t x = (corner & 1) ? hi[0] : lo[0];
                int32_t y = (corner & 2) ? hi[1] : lo[1];
                int32_t z = (corner & 4) ? hi[2] : lo[2];
                double w = ((corner & 1) ? f[0] : 1.0 - f[0]) * ((corner & 2) ? f[1] : 1.0 - f[1]) *
                           ((corner & 4) ? f[2] : 1.0 - f[2]);
                val += w * rf[c * ng + ((size_t)z * gn[1] + y) * gn[0] + x];
            }
            disp[c * nvox + v] = val - p[c];
        }
    }
    free(rf);
    return OR_OK;
}
