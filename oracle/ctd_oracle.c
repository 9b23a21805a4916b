/*
 * ctd_oracle.c -- CPU oracle for the gCTD photon transport (TEST INFRASTRUCTURE).
 *
 * Plain, slow restatement of arXiv:1109.3266 used only by the tests, the smoke
 * check and the CPU-baseline leg of the benchmark.  Nothing in the product
 * library includes, links or calls this file; the two share no source.
 *
 * Readings of the paper that the code below takes (the paper leaves them open):
 *   - attenuation data are linear interpolation in E of closed forms sampled at
 *     integer-keV nodes (Sec. 2.2.7 item 3); the node grid's floor is the
 *     absorption energy (Sec. 3.1);
 *   - photoelectric per formula unit 1e-2 Z^4 / E_MeV^3 in microbarn,
 *     Rayleigh per formula unit 1.565e-5 Z^2 / E_MeV^2 in barn, Compton
 *     = free-electron Klein-Nishina total per electron times electrons per gram;
 *   - Rayleigh form factor F^2(q^2) ~ exp(-q^2 / q0^2) (or 1, Thomson), or the
 *     independent-atom molecular form factor sum_i n_i F_Zi^2 with a screened
 *     hydrogenic atom per element (Thomas-Fermi radius), whose Rayleigh total is
 *     then the integral of Eq. 1 by composite Simpson;
 *   - Waller-Hartree Compton (Eq. 2 with S(q)): S(q)/Z = 1 - exp(-q^2 / sq0^2)
 *     with q^2 = 2 k^2 (1 - cos theta), k = E / hc, the same momentum transfer as
 *     the form factor; its total is the integral of Eq. 2 by composite Simpson;
 *   - random numbers: Philox4x32-10 keyed by the 64-bit seed, counter
 *     (history lo, history hi, step, stream).
 */
#define _GNU_SOURCE
#include "ctd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- physical constants (CODATA 2018) ---- */
#define OR_MEC2 510.99895          /* electron rest energy, keV            */
#define OR_R0 2.8179403262e-13     /* classical electron radius, cm        */
#define OR_NA 6.02214076e23        /* Avogadro, 1/mol                       */
#define OR_HC 12.398419843320026   /* h c, keV Angstrom                     */
#define OR_PI 3.141592653589793
#define OR_UBARN 1.0e-30           /* microbarn, cm^2                       */
#define OR_BARN 1.0e-24            /* barn, cm^2                            */
#define OR_PE_COEF 1.0e-2          /* photoelectric coefficient (microbarn) */
#define OR_RAY_COEF 1.565e-5       /* Rayleigh coefficient (barn MeV^2)     */
#define OR_CDF_POINTS 20000        /* mu intervals of the numeric cdf       */
#define OR_MAX_TRIALS 1000         /* rejection loops give up after this    */
#define OR_MAX_TRIALS_WH (1u << 20) /* Waller-Hartree keeps about a(1-mu) of KN draws at low E */
#define OR_MAX_STEPS 100000000u    /* Woodcock steps per history            */
#define OR_BOHR 0.529177210903     /* Bohr radius, Angstrom                 */
#define OR_TF 0.88534138           /* Thomas-Fermi radius / (a0 Z^-1/3): (3 pi / 4)^(2/3) / 2 */

enum { OR_STREAM_TRANSPORT = 0, OR_STREAM_SOURCE = 1, OR_STREAM_EXACT = 2, OR_STREAM_SAMPLER = 3, OR_STREAM_MH = 4 };

/* ===================================================================== */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.2): ten rounds */
/* of two 32x32->64 multiplications, xor with the key, and a Weyl key step. */
/* ===================================================================== */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on (0,1): (2*(x>>9)+1) * 2^-24, exact in binary32 and binary64. */
double or_uniform(uint32_t x) { return (double)(2u * (x >> 9) + 1u) * 0x1p-24; }
static float or_uniform_f(uint32_t x) { return (float)(2u * (x >> 9) + 1u) * 0x1p-24f; }

static void or_block(uint64_t seed, uint64_t h, uint32_t step, uint32_t stream, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)h, (uint32_t)(h >> 32), step, stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* ===================================================================== */
/* Single-precision logarithm and sincos used by the binary32 method.     */
/* log: write u = 2^e m with m in (sqrt(1/2), sqrt(2)], then               */
/* ln m = 2 atanh(s), s = (m-1)/(m+1), by the atanh Taylor series to s^11. */
/* sincos of 2 pi t: exact reduction of t in turns to a quarter-turn       */
/* offset r in [-1/8, 1/8], Taylor series of sin and cos of 2 pi r.        */
/* ===================================================================== */
float or_log_f32(float u)
{
    union { float f; uint32_t i; } b;
    b.f = u;
    int e = (int)((b.i >> 23) & 0xffu) - 127;
    b.i = (b.i & 0x7fffffu) | 0x3f800000u;
    float m = b.f;
    if (m > 0x1.6a09e6p+0f) { m = m * 0.5f; e = e + 1; }
    float f = m - 1.0f;
    float s = f / (2.0f + f);
    float z = s * s;
    float p = fmaf(z, 0x1.745d18p-4f, 0x1.c71c72p-4f);
    p = fmaf(z, p, 0x1.24924ap-3f);
    p = fmaf(z, p, 0x1.99999ap-3f);
    p = fmaf(z, p, 0x1.555556p-2f);
    float r = z * p;
    float s2 = s + s;
    float lnm = fmaf(s2, r, s2);
    float ef = (float)e;
    return fmaf(ef, 0x1.62e430p-1f, fmaf(ef, -0x1.05c610p-29f, lnm));
}

void or_sincos_turns_f32(float t, float *c, float *s)
{
    float fl = floorf(t);
    float w = t - fl;                     /* exact: drops the integer bits */
    int q = (int)(w * 4.0f);
    float r = w - (float)q * 0.25f;       /* exact */
    if (r > 0.125f) { r = r - 0.25f; q = q + 1; }
    float x = r * 0x1.921fb6p+2f;         /* 2 pi r */
    float x2 = x * x;
    float ps = fmaf(x2, 0x1.71de3ap-19f, -0x1.a01a02p-13f);
    ps = fmaf(x2, ps, 0x1.111112p-7f);
    ps = fmaf(x2, ps, -0x1.555556p-3f);
    float sn = fmaf(x * x2, ps, x);
    float pc = fmaf(x2, -0x1.27e4fcp-22f, 0x1.a01a02p-16f);
    pc = fmaf(x2, pc, -0x1.6c16c2p-10f);
    pc = fmaf(x2, pc, 0x1.555556p-5f);
    pc = fmaf(x2, pc, -0.5f);
    float cs = fmaf(x2, pc, 1.0f);
    switch (q & 3) {
    case 0: *c = cs; *s = sn; break;
    case 1: *c = -sn; *s = cs; break;
    case 2: *c = -cs; *s = -sn; break;
    default: *c = sn; *s = -cs; break;
    }
}

/* binary64 -> binary32 by truncating the significand to 23 bits (round toward
 * zero); magnitudes below 2^-126 give 0. */
static float or_trunc32(double d)
{
    uint64_t b;
    memcpy(&b, &d, sizeof b);
    uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    uint32_t ex = (hi >> 20) & 0x7ffu;
    if (ex < 897u) return 0.0f;
    uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    uint32_t f = (hi & 0x80000000u) | (((ex - 896u) & 0xffu) << 23) | m;
    float r;
    memcpy(&r, &f, sizeof r);
    return r;
}

void or_eval_log_f32(const float *u, float *out, size_t n)
{
    for (size_t i = 0; i < n; ++i) out[i] = or_log_f32(u[i]);
}

void or_eval_uniform_f32(const uint32_t *x, float *out, size_t n)
{
    for (size_t i = 0; i < n; ++i) out[i] = or_uniform_f(x[i]);
}

void or_eval_sincos_f32(const float *t, float *c, float *s, size_t n)
{
    for (size_t i = 0; i < n; ++i) or_sincos_turns_f32(t[i], &c[i], &s[i]);
}

/* ===================================================================== */
/* Closed-form cross sections (Sec. 2.1; Eq. 2 with S = 1 for Compton).    */
/* ===================================================================== */
double or_sigma_kn(double e_kev)
{
    /* Klein-Nishina total cross section per electron, cm^2 */
    double k = e_kev / OR_MEC2;
    double a = 1.0 + 2.0 * k;
    double l = log1p(2.0 * k);
    double t1 = ((1.0 + k) / (k * k)) * ((2.0 * (1.0 + k)) / a - l / k);
    double t2 = l / (2.0 * k);
    double t3 = (1.0 + 3.0 * k) / (a * a);
    return 2.0 * OR_PI * OR_R0 * OR_R0 * ((t1 + t2) - t3);
}

double or_mu_compton(const or_material *m, double e_kev)
{
    return (OR_NA * m->z_over_a) * or_sigma_kn(e_kev);
}

double or_mu_pe(const or_material *m, double e_kev)
{
    double em = e_kev / 1000.0;
    double z2 = m->z_eff * m->z_eff;
    double sigma = OR_PE_COEF * (z2 * z2) / (em * em * em);   /* microbarn per formula unit */
    return ((sigma * OR_UBARN) * OR_NA) / m->a_mol;
}

double or_mu_rayleigh(const or_material *m, double e_kev)
{
    double em = e_kev / 1000.0;
    double z2 = m->z_eff * m->z_eff;
    double sigma = OR_RAY_COEF * z2 / (em * em);              /* barn per formula unit */
    return ((sigma * OR_BARN) * OR_NA) / m->a_mol;
}

/* Eq. 2 up to the factor r0^2/2: the Klein-Nishina density in mu = cos theta
 * times S(q)/Z = 1 - exp(-a (1 - mu)), a = 2 k^2 / sq0^2 (a <= 0: S/Z = 1). */
static double or_pdf_wh(double k, double a, double mu)
{
    double e = 1.0 / (1.0 + k * (1.0 - mu));
    double kn = (e * e) * ((e + 1.0 / e) - (1.0 - mu * mu));
    if (a <= 0.0) return kn;
    return kn * (-expm1(-a * (1.0 - mu)));
}

static double or_wh_a(double e_kev, double sq0)
{
    double kr = e_kev / OR_HC;
    return sq0 > 0.0 ? (2.0 * kr * kr) / (sq0 * sq0) : 0.0;
}

double or_sigma_wh(double e_kev, double sq0)
{
    const int M = OR_CDF_POINTS;
    double k = e_kev / OR_MEC2;
    double a = or_wh_a(e_kev, sq0);
    /* Simpson weights 1, 4, 2, ..., 4, 1 on mu_n = (2n - M)/M, h = 2/M */
    double odd = 0.0, even = 0.0;
    for (int n = 1; n < M; ++n) {
        double mu = (double)(2 * n - M) / (double)M;
        if (n & 1) odd += or_pdf_wh(k, a, mu);
        else even += or_pdf_wh(k, a, mu);
    }
    double ends = or_pdf_wh(k, a, -1.0) + or_pdf_wh(k, a, 1.0);
    double integral = ((2.0 / (double)M) / 3.0) * (ends + (4.0 * odd + 2.0 * even));
    /* dsigma/dOmega = (r0^2/2) pdf, dOmega = 2 pi dmu */
    return (OR_PI * OR_R0 * OR_R0) * integral;
}

double or_mu_compton_wh(const or_material *m, double e_kev)
{
    return (OR_NA * m->z_over_a) * or_sigma_wh(e_kev, m->sq0);
}

/* Independent-atom Rayleigh form factor.  A screened hydrogenic atom, electron
 * density Z exp(-2 r / a) / (pi a^3), has the form factor F(Q) = Z / (1 + (Q a/2)^2)^2
 * at momentum transfer Q = 4 pi x, x = sin(theta/2) / lambda; the screening length
 * is the Thomas-Fermi radius a = 0.8853 a0 Z^(-1/3).  So F^2 = Z^2 / (1 + c x^2)^4
 * with c = (2 pi a)^2.  The molecule's F^2 is the sum over its atoms (no
 * interference between them). */
static double or_ff_width(int z)
{
    double a = (OR_TF * OR_BOHR) / cbrt((double)z);
    double w = (2.0 * OR_PI) * a;
    return w * w;
}

static double or_ff_z2(double z, double c, double x2)
{
    double g = 1.0 / (1.0 + c * x2);
    double f = z * (g * g);
    return f * f;
}

double or_ff_atom2(int z, double x2)
{
    return or_ff_z2((double)z, or_ff_width(z), x2);
}

/* F^2_mol from the elements' widths c[i] */
static double or_ff_sum2(const or_material *m, const double *c, double x2)
{
    double s = 0.0;
    for (int i = 0; i < m->n_el; ++i) s += m->el_n[i] * or_ff_z2((double)m->el_z[i], c[i], x2);
    return s;
}

double or_ff_mol2(const or_material *m, double x2)
{
    double c[OR_MAX_ELEMENTS];
    for (int i = 0; i < m->n_el; ++i) c[i] = or_ff_width(m->el_z[i]);
    return or_ff_sum2(m, c, x2);
}

/* Eq. 1 up to r0^2/2: (1 + mu^2) F^2_mol(x), x^2 = k^2 (1 - mu) / 2, k = E/hc in 1/Angstrom */
static double or_pdf_rayleigh_iaa(const or_material *m, const double *c, double kr, double mu)
{
    double x2 = ((kr * kr) * (1.0 - mu)) * 0.5;
    return (1.0 + mu * mu) * or_ff_sum2(m, c, x2);
}

double or_sigma_rayleigh_iaa(const or_material *m, double e_kev)
{
    const int M = OR_CDF_POINTS;
    double kr = e_kev / OR_HC;
    double c[OR_MAX_ELEMENTS];
    for (int i = 0; i < m->n_el; ++i) c[i] = or_ff_width(m->el_z[i]);
    /* Simpson weights 1, 4, 2, ..., 4, 1 on mu_n = (2n - M)/M, h = 2/M */
    double odd = 0.0, even = 0.0;
    for (int n = 1; n < M; ++n) {
        double mu = (double)(2 * n - M) / (double)M;
        if (n & 1) odd += or_pdf_rayleigh_iaa(m, c, kr, mu);
        else even += or_pdf_rayleigh_iaa(m, c, kr, mu);
    }
    double ends = or_pdf_rayleigh_iaa(m, c, kr, -1.0) + or_pdf_rayleigh_iaa(m, c, kr, 1.0);
    double integral = ((2.0 / (double)M) / 3.0) * (ends + (4.0 * odd + 2.0 * even));
    /* dsigma/dOmega = (r0^2/2) (1 + mu^2) F^2, dOmega = 2 pi dmu */
    return (OR_PI * OR_R0 * OR_R0) * integral;
}

double or_mu_rayleigh_iaa(const or_material *m, double e_kev)
{
    return (or_sigma_rayleigh_iaa(m, e_kev) * OR_NA) / m->a_mol;
}

/* ===================================================================== */
/* Largest-remainder allocation of n histories to spectrum bins           */
/* (Sec. 2.2.5: histories distributed to 1 keV intervals by the spectrum). */
/* ===================================================================== */
int or_allocate(uint64_t n, int nbins, const double *w, uint64_t *out)
{
    if (nbins <= 0) return -1;
    double total = 0.0;
    for (int j = 0; j < nbins; ++j) {
        if (!(w[j] >= 0.0) || !isfinite(w[j])) return -1;
        total += w[j];
    }
    if (!(total > 0.0) || !isfinite(total)) return -1;
    double *frac = (double *)malloc(sizeof(double) * (size_t)nbins);
    if (!frac) return -1;
    uint64_t given = 0;
    for (int j = 0; j < nbins; ++j) {
        double q = (double)n * w[j] / total;
        double fl = floor(q);
        out[j] = (uint64_t)fl;
        frac[j] = q - fl;
        given += out[j];
    }
    /* hand out the remainder one at a time: largest fraction first, ties to the lower bin */
    while (given < n) {
        int best = -1;
        for (int j = 0; j < nbins; ++j) {
            if (w[j] <= 0.0) continue;
            if (best < 0 || frac[j] > frac[best]) best = j;
        }
        if (best < 0) break;
        out[best] += 1;
        frac[best] = -1.0;
        given += 1;
    }
    /* the floors can overshoot only through rounding of q; take back from the smallest fractions */
    while (given > n) {
        int best = -1;
        for (int j = nbins - 1; j >= 0; --j) {
            if (out[j] == 0) continue;
            if (best < 0 || frac[j] < frac[best]) best = j;
        }
        if (best < 0) break;
        out[best] -= 1;
        frac[best] = 2.0;
        given -= 1;
    }
    free(frac);
    return given == n ? 0 : -1;
}

/* ===================================================================== */
/* R and C surfaces (Sec. 2.2.2, Sec. 2.2.3): pdf on an even mu grid,      */
/* cumulative trapezoid cdf, inverse at evenly spaced zeta by linear       */
/* interpolation, one row per node energy.                                */
/* ===================================================================== */
static double or_pdf_kn(double k, double mu)
{
    /* Eq. 2 with S = 1, up to a constant: (E'/E)^2 (E'/E + E/E' - sin^2 theta) */
    double e = 1.0 / (1.0 + k * (1.0 - mu));
    return (e * e) * ((e + 1.0 / e) - (1.0 - mu * mu));
}

static double or_pdf_rayleigh(double a, double mu)
{
    /* Eq. 1 up to a constant: (1 + cos^2 theta) F^2, F^2 = exp(-q^2/q0^2), q^2 = 2k^2(1-mu) */
    if (a <= 0.0) return 1.0 + mu * mu;
    return (1.0 + mu * mu) * exp(-a * (1.0 - mu));
}

static void or_invert_row(const double *cdf, int n_zeta, double *row)
{
    const int M = OR_CDF_POINTS;
    double total = cdf[M];
    int n = 0;
    row[0] = -1.0;
    for (int i = 1; i < n_zeta - 1; ++i) {
        double target = ((double)i / (double)(n_zeta - 1)) * total;
        while (n < M - 1 && cdf[n + 1] <= target) ++n;
        double mu_n = (double)(2 * n - M) / (double)M;
        double mu_n1 = (double)(2 * (n + 1) - M) / (double)M;
        row[i] = mu_n + ((target - cdf[n]) / (cdf[n + 1] - cdf[n])) * (mu_n1 - mu_n);
    }
    row[n_zeta - 1] = 1.0;
}

/* kind 0: Klein-Nishina C surface; 1: Rayleigh R surface of width q0;
 * 2: Waller-Hartree C surface of scattering-function width q0;
 * 3: Rayleigh R surface with the independent-atom form factor of material m */
static void or_build_surface(int kind, double q0, const or_material *m, int e_min, int n_e, int n_zeta, double *out)
{
    const int M = OR_CDF_POINTS;
    double *pdf = (double *)malloc(sizeof(double) * (size_t)(M + 1));
    double *cdf = (double *)malloc(sizeof(double) * (size_t)(M + 1));
    double c[OR_MAX_ELEMENTS];
    if (kind == 3)
        for (int i = 0; i < m->n_el; ++i) c[i] = or_ff_width(m->el_z[i]);
    for (int j = 0; j < n_e; ++j) {
        double e = (double)(e_min + j);
        double k = e / OR_MEC2;
        double kr = e / OR_HC;
        double a = q0 > 0.0 ? (2.0 * kr * kr) / (q0 * q0) : 0.0;
        for (int n = 0; n <= M; ++n) {
            double mu = (double)(2 * n - M) / (double)M;
            pdf[n] = kind == 0   ? or_pdf_kn(k, mu)
                     : kind == 1 ? or_pdf_rayleigh(a, mu)
                     : kind == 2 ? or_pdf_wh(k, a, mu)
                                 : or_pdf_rayleigh_iaa(m, c, kr, mu);
        }
        cdf[0] = 0.0;
        for (int n = 1; n <= M; ++n) cdf[n] = cdf[n - 1] + (pdf[n - 1] + pdf[n]);
        or_invert_row(cdf, n_zeta, out + (size_t)j * (size_t)n_zeta);
    }
    free(pdf);
    free(cdf);
}

void or_build_kn_surface(int e_min, int n_e, int n_zeta, double *out)
{
    or_build_surface(0, 0.0, NULL, e_min, n_e, n_zeta, out);
}

void or_build_rayleigh_surface(double q0, int e_min, int n_e, int n_zeta, double *out)
{
    or_build_surface(1, q0, NULL, e_min, n_e, n_zeta, out);
}

void or_build_wh_surface(double sq0, int e_min, int n_e, int n_zeta, double *out)
{
    or_build_surface(2, sq0, NULL, e_min, n_e, n_zeta, out);
}

void or_build_rayleigh_iaa_surface(const or_material *m, int e_min, int n_e, int n_zeta, double *out)
{
    or_build_surface(3, 0.0, m, e_min, n_e, n_zeta, out);
}

/* ===================================================================== */
/* Fluence map (Sec. 2.2.4): the beamlet index I with probability f_I.    */
/* Alias table: Walker's method built with Vose's two work lists.         */
/* ===================================================================== */
int or_alias_build(int n, const double *f, uint32_t *thr, int32_t *alias)
{
    if (n <= 0) return -1;
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(f[i] >= 0.0) || !isfinite(f[i])) return -1;
        total += f[i];
    }
    if (!(total > 0.0) || !isfinite(total)) return -1;
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    int *small = (int *)malloc(sizeof(int) * (size_t)n);
    int *large = (int *)malloc(sizeof(int) * (size_t)n);
    int ns = 0, nl = 0;
    /* scaled probabilities n f_i / total; columns below 1 borrow from columns above */
    for (int i = 0; i < n; ++i) {
        p[i] = (f[i] * (double)n) / total;
        if (p[i] < 1.0) small[ns++] = i;
        else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        int l = small[--ns], g = large[--nl];
        thr[l] = (uint32_t)(p[l] * 4294967296.0);
        alias[l] = g;
        p[g] = (p[g] + p[l]) - 1.0;
        if (p[g] < 1.0) small[ns++] = g;
        else large[nl++] = g;
    }
    /* what is left is 1 up to rounding */
    while (nl > 0) { int g = large[--nl]; thr[g] = 0xffffffffu; alias[g] = g; }
    while (ns > 0) { int l = small[--ns]; thr[l] = 0xffffffffu; alias[l] = l; }
    free(p); free(small); free(large);
    return 0;
}

static uint32_t or_alias_draw(int n_f, const uint32_t *thr, const int32_t *alias, uint32_t x, uint32_t y)
{
    uint32_t k = (uint32_t)(((uint64_t)x * (uint64_t)(uint32_t)n_f) >> 32);
    return y < thr[k] ? k : (uint32_t)alias[k];
}

void or_alias_counts(int n_f, const uint32_t *thr, const int32_t *alias, uint64_t n, uint64_t seed,
                     uint64_t *counts)
{
    for (int i = 0; i < n_f; ++i) counts[i] = 0;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t b[4];
        or_block(seed, i, 1, OR_STREAM_SOURCE, b);
        counts[or_alias_draw(n_f, thr, alias, b[0], b[1])]++;
    }
}

void or_mh_counts(int n_f, const double *f, int i0, uint64_t n, uint64_t seed, uint64_t *counts)
{
    for (int i = 0; i < n_f; ++i) counts[i] = 0;
    int last = i0;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t b[4];
        or_block(seed, i, 0, OR_STREAM_MH, b);
        /* 1. trial beamlet J uniform; 2. zeta uniform; 3. keep J if zeta < f_J / f_last */
        int j = (int)(((uint64_t)b[0] * (uint64_t)(uint32_t)n_f) >> 32);
        double zeta = or_uniform(b[1]);
        int cur = zeta < f[j] / f[last] ? j : last;
        counts[cur]++;
        last = cur;
    }
}

/* Algorithm A1 as the paper runs it on a GPU: one chain per thread.  Chain c of
 * `chains` takes particles [n c / chains, n (c + 1) / chains), starts at beamlet
 * i0 and draws particle i from Philox block (i, 0, stream 4), as the single chain
 * does; the counts of all chains are summed.  chains = 1 is or_mh_counts. */
void or_mh_chains(int n_f, const double *f, int i0, uint64_t n, uint64_t seed, uint64_t chains, uint64_t *counts)
{
    for (int i = 0; i < n_f; ++i) counts[i] = 0;
    for (uint64_t c = 0; c < chains; ++c) {
        uint64_t lo = (n / chains) * c + (c < n % chains ? c : n % chains);
        uint64_t len = n / chains + (c < n % chains ? 1 : 0);
        int last = i0;
        for (uint64_t i = lo; i < lo + len; ++i) {
            uint32_t b[4];
            or_block(seed, i, 0, OR_STREAM_MH, b);
            int j = (int)(((uint64_t)b[0] * (uint64_t)(uint32_t)n_f) >> 32);
            double zeta = or_uniform(b[1]);
            int cur = zeta < f[j] / f[last] ? j : last;
            counts[cur]++;
            last = cur;
        }
    }
}

/* ===================================================================== */
/* Set-up: tables, majorant, surfaces, batch and bin offsets.            */
/* ===================================================================== */
struct or_setup {
    or_problem p;
    int prec;
    int n_e;
    double *tab64; float *tab32;   /* [n_mat][n_e][3]: PE, PE+C, PE+C+R mass attenuation */
    double *mm64; float *mm32;     /* [n_e] majorant mu_max(E), 1/cm (Sec. 2.1)         */
    int n_cs;                      /* C surfaces: 1 (Klein-Nishina) or n_mat (Waller-Hartree) */
    double *cs64; float *cs32;     /* [n_cs][n_e][n_zeta] C surfaces                     */
    double *rs64; float *rs32;     /* [n_mat][n_e][n_zeta] R surfaces                    */
    uint64_t n_lo, n_rem;          /* batch sizes: first n_rem batches hold n_lo + 1     */
    uint64_t *pref_big, *pref_small; /* [nbins + 1] bin start offsets inside a batch     */
    /* geometry in both precisions */
    double bx0, by0, bz0, bx1, by1, bz1, ix, iy, iz;
    float fbx0, fby0, fbz0, fbx1, fby1, fbz1, fix, fiy, fiz;
    double *cb64, *sb64; float *cb32, *sb32; /* projection angle cos/sin */
    double *zb64; float *zb32;     /* projection source height (helical trajectory)       */
    float fz0, fdz;                /* z0 and z1 - z0 in binary32                         */
    int fl_n;                      /* beamlets (0: no fluence map)                       */
    uint32_t *fl_thr; int32_t *fl_alias;
    double fl_du, fl_dv; float fl_fdu, fl_fdv;   /* beamlet size at the centre plane  */
};

static void or_setup_free(or_setup *s)
{
    if (!s) return;
    free(s->tab64); free(s->tab32); free(s->mm64); free(s->mm32);
    free(s->cs64); free(s->cs32); free(s->rs64); free(s->rs32);
    free(s->pref_big); free(s->pref_small);
    free(s->cb64); free(s->sb64); free(s->cb32); free(s->sb32); free(s->zb64); free(s->zb32);
    free(s->fl_thr); free(s->fl_alias);
    free(s);
}

void or_setup_destroy(or_setup *s) { or_setup_free(s); }

static or_setup *or_setup_create(const or_problem *p, int prec)
{
    if (p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || p->n_mat <= 0 || p->nbins <= 0) return NULL;
    if (p->e_max <= p->e_min || p->e_min <= 0 || p->n_zeta < 2 || p->n_batches <= 0) return NULL;
    if (!(p->majorant_scale >= 1.0)) return NULL;
    if (p->compton != OR_COMPTON_KN && p->compton != OR_COMPTON_WH) return NULL;
    for (int j = 0; j < p->nbins; ++j)
        if (!(p->e_lo[j] >= p->e_min && p->e_hi[j] <= p->e_max && p->e_hi[j] >= p->e_lo[j])) return NULL;
    or_setup *s = (or_setup *)calloc(1, sizeof(or_setup));
    if (!s) return NULL;
    s->p = *p;
    s->prec = prec;
    int n_e = p->e_max - p->e_min + 1;
    int nm = p->n_mat, nz = p->n_zeta;
    s->n_e = n_e;
    size_t nvox = (size_t)p->nx * (size_t)p->ny * (size_t)p->nz;
    s->tab64 = (double *)malloc(sizeof(double) * (size_t)nm * n_e * 3);
    s->tab32 = (float *)malloc(sizeof(float) * (size_t)nm * n_e * 3);
    s->mm64 = (double *)malloc(sizeof(double) * n_e);
    s->mm32 = (float *)malloc(sizeof(float) * n_e);
    s->n_cs = p->compton == OR_COMPTON_WH ? nm : 1;
    s->cs64 = (double *)malloc(sizeof(double) * (size_t)s->n_cs * n_e * nz);
    s->cs32 = (float *)malloc(sizeof(float) * (size_t)s->n_cs * n_e * nz);
    s->rs64 = (double *)malloc(sizeof(double) * (size_t)nm * n_e * nz);
    s->rs32 = (float *)malloc(sizeof(float) * (size_t)nm * n_e * nz);
    double *rho_max = (double *)calloc((size_t)nm, sizeof(double));
    int *present = (int *)calloc((size_t)nm, sizeof(int));
    for (size_t v = 0; v < nvox; ++v) {
        int m = p->mat[v];
        if (m >= nm) { free(rho_max); free(present); or_setup_free(s); return NULL; }
        double r = (double)p->rho[v];
        if (!(r >= 0.0)) { free(rho_max); free(present); or_setup_free(s); return NULL; }
        if (!present[m] || r > rho_max[m]) rho_max[m] = r;
        present[m] = 1;
    }
    /* node tables: cumulative mass attenuation per material */
    for (int m = 0; m < nm; ++m) {
        for (int j = 0; j < n_e; ++j) {
            double e = (double)(p->e_min + j);
            double pe = or_mu_pe(&p->mats[m], e);
            double c = p->compton == OR_COMPTON_WH ? or_mu_compton_wh(&p->mats[m], e) : or_mu_compton(&p->mats[m], e);
            double r = p->mats[m].n_el > 0 ? or_mu_rayleigh_iaa(&p->mats[m], e) : or_mu_rayleigh(&p->mats[m], e);
            size_t o = ((size_t)m * n_e + j) * 3;
            s->tab64[o + 0] = pe;
            s->tab64[o + 1] = pe + c;
            s->tab64[o + 2] = (pe + c) + r;
            for (int q = 0; q < 3; ++q) s->tab32[o + q] = (float)s->tab64[o + q];
        }
    }
    /* majorant mu_max(E): the largest total attenuation over the volume (Sec. 2.1) */
    for (int j = 0; j < n_e; ++j) {
        double best = 0.0;
        for (int m = 0; m < nm; ++m) {
            if (!present[m]) continue;
            double v = rho_max[m] * s->tab64[((size_t)m * n_e + j) * 3 + 2];
            if (v > best) best = v;
        }
        s->mm64[j] = p->majorant_scale * best;
        s->mm32[j] = (float)s->mm64[j];
    }
    free(rho_max);
    free(present);
    /* surfaces */
    if (p->compton == OR_COMPTON_WH) {
        for (int m = 0; m < nm; ++m)
            or_build_wh_surface(p->mats[m].sq0, p->e_min, n_e, nz, s->cs64 + (size_t)m * n_e * nz);
    } else {
        or_build_kn_surface(p->e_min, n_e, nz, s->cs64);
    }
    for (size_t i = 0; i < (size_t)s->n_cs * n_e * nz; ++i) s->cs32[i] = (float)s->cs64[i];
    for (int m = 0; m < nm; ++m) {
        double *dst = s->rs64 + (size_t)m * n_e * nz;
        if (p->mats[m].n_el > 0) or_build_rayleigh_iaa_surface(&p->mats[m], p->e_min, n_e, nz, dst);
        else or_build_rayleigh_surface(p->mats[m].q0, p->e_min, n_e, nz, dst);
        for (size_t i = 0; i < (size_t)n_e * nz; ++i) s->rs32[(size_t)m * n_e * nz + i] = (float)dst[i];
    }
    /* batches (Sec. 2.2.1) and the stratified allocation inside each (Sec. 2.2.5) */
    s->n_lo = p->n_hist / (uint64_t)p->n_batches;
    s->n_rem = p->n_hist % (uint64_t)p->n_batches;
    s->pref_big = (uint64_t *)calloc((size_t)p->nbins + 1, sizeof(uint64_t));
    s->pref_small = (uint64_t *)calloc((size_t)p->nbins + 1, sizeof(uint64_t));
    uint64_t *tmp = (uint64_t *)calloc((size_t)p->nbins, sizeof(uint64_t));
    if (or_allocate(s->n_lo + 1, p->nbins, p->w, tmp) != 0) { free(tmp); or_setup_free(s); return NULL; }
    for (int j = 0; j < p->nbins; ++j) s->pref_big[j + 1] = s->pref_big[j] + tmp[j];
    if (or_allocate(s->n_lo, p->nbins, p->w, tmp) != 0) { free(tmp); or_setup_free(s); return NULL; }
    for (int j = 0; j < p->nbins; ++j) s->pref_small[j + 1] = s->pref_small[j] + tmp[j];
    free(tmp);
    /* box, centred at the origin, half-open voxels */
    double hx = (double)p->nx * p->dx / 2.0, hy = (double)p->ny * p->dy / 2.0, hz = (double)p->nz * p->dz / 2.0;
    s->bx0 = -hx; s->by0 = -hy; s->bz0 = -hz; s->bx1 = hx; s->by1 = hy; s->bz1 = hz;
    s->ix = 1.0 / p->dx; s->iy = 1.0 / p->dy; s->iz = 1.0 / p->dz;
    s->fbx0 = (float)s->bx0; s->fby0 = (float)s->by0; s->fbz0 = (float)s->bz0;
    s->fbx1 = (float)s->bx1; s->fby1 = (float)s->by1; s->fbz1 = (float)s->bz1;
    s->fix = (float)s->ix; s->fiy = (float)s->iy; s->fiz = (float)s->iz;
    /* fluence map: alias table over the beamlets */
    if (p->fl_nu > 0) {
        if (p->fl_nv <= 0 || !p->fl_f || (int64_t)p->fl_nu * p->fl_nv > (1 << 24)) { or_setup_free(s); return NULL; }
        s->fl_n = p->fl_nu * p->fl_nv;
        s->fl_thr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)s->fl_n);
        s->fl_alias = (int32_t *)malloc(sizeof(int32_t) * (size_t)s->fl_n);
        if (or_alias_build(s->fl_n, p->fl_f, s->fl_thr, s->fl_alias) != 0) { or_setup_free(s); return NULL; }
        s->fl_du = (p->u_hi - p->u_lo) / (double)p->fl_nu;
        s->fl_dv = (p->v_hi - p->v_lo) / (double)p->fl_nv;
        s->fl_fdu = (float)s->fl_du;
        s->fl_fdv = (float)s->fl_dv;
    }
    /* projection angles beta_k = arc0 + (arc1 - arc0) k / n_proj */
    int np = p->n_proj > 0 ? p->n_proj : 1;
    s->cb64 = (double *)malloc(sizeof(double) * np); s->sb64 = (double *)malloc(sizeof(double) * np);
    s->cb32 = (float *)malloc(sizeof(float) * np); s->sb32 = (float *)malloc(sizeof(float) * np);
    s->zb64 = (double *)malloc(sizeof(double) * np); s->zb32 = (float *)malloc(sizeof(float) * np);
    for (int k = 0; k < np; ++k) {
        double b = p->arc0 + (p->arc1 - p->arc0) * (double)k / (double)np;
        s->cb64[k] = cos(b); s->sb64[k] = sin(b);
        s->cb32[k] = (float)s->cb64[k]; s->sb32[k] = (float)s->sb64[k];
        /* helical: the height moves with the angle, z_k = z0 + (z1 - z0) k / n_proj */
        s->zb64[k] = p->z0 + (p->z1 - p->z0) * (double)k / (double)np;
        s->zb32[k] = (float)s->zb64[k];
    }
    s->fz0 = (float)p->z0;
    s->fdz = (float)(p->z1 - p->z0);
    return s;
}

or_setup *or_setup_create_f64(const or_problem *p) { return or_setup_create(p, 64); }
or_setup *or_setup_create_f32(const or_problem *p) { return or_setup_create(p, 32); }

int or_setup_sizes(const or_setup *s, int *n_e, int *n_zeta, int *n_mat)
{
    *n_e = s->n_e; *n_zeta = s->p.n_zeta; *n_mat = s->p.n_mat;
    return 0;
}

void or_setup_tables(const or_setup *s, double *mu_cum, double *mu_max)
{
    size_t nt = (size_t)s->p.n_mat * s->n_e * 3;
    for (size_t i = 0; i < nt; ++i) mu_cum[i] = s->prec == 32 ? (double)s->tab32[i] : s->tab64[i];
    for (int j = 0; j < s->n_e; ++j) mu_max[j] = s->prec == 32 ? (double)s->mm32[j] : s->mm64[j];
}

void or_setup_surfaces(const or_setup *s, double *c_surf, double *r_surf)
{
    size_t nc = (size_t)s->n_e * s->p.n_zeta;
    for (size_t i = 0; i < (size_t)s->n_cs * nc; ++i) c_surf[i] = s->prec == 32 ? (double)s->cs32[i] : s->cs64[i];
    size_t nr = (size_t)s->p.n_mat * nc;
    for (size_t i = 0; i < nr; ++i) r_surf[i] = s->prec == 32 ? (double)s->rs32[i] : s->rs64[i];
}

/* history index -> (batch, bin) */
static int or_bin_of(const or_setup *s, uint64_t h, uint64_t *batch_size)
{
    uint64_t big = s->n_rem * (s->n_lo + 1);
    uint64_t local;
    const uint64_t *pref;
    if (h < big) {
        local = h % (s->n_lo + 1);
        pref = s->pref_big;
        *batch_size = s->n_lo + 1;
    } else {
        local = (h - big) % s->n_lo;
        pref = s->pref_small;
        *batch_size = s->n_lo;
    }
    int j = 0;
    while (j < s->p.nbins - 1 && pref[j + 1] <= local) ++j;
    return j;
}

/* ===================================================================== */
/* Exact angular samplers (f64 only): Kahn's rejection for Klein-Nishina,  */
/* and for Rayleigh sampling of F^2 followed by rejection on (1+mu^2)/2    */
/* (the generalized rejection the paper describes in Sec. 2.2.2).          */
/* ===================================================================== */
static double or_exact_kn(double e_kev, uint64_t seed, uint64_t h, uint32_t step, int *ok)
{
    double k = e_kev / OR_MEC2;
    double p1 = (1.0 + 2.0 * k) / (9.0 + 2.0 * k);
    for (uint32_t t = 0; t < OR_MAX_TRIALS; ++t) {
        uint32_t b[4];
        or_block(seed, h, step, OR_STREAM_EXACT | (t << 8), b);
        double r1 = or_uniform(b[0]), r2 = or_uniform(b[1]), r3 = or_uniform(b[2]);
        if (r1 <= p1) {
            double x = 1.0 + 2.0 * k * r2;                     /* x = E/E' */
            if (r3 <= 4.0 * (1.0 / x - 1.0 / (x * x))) { *ok = 1; return 1.0 - (x - 1.0) / k; }
        } else {
            double x = (1.0 + 2.0 * k) / (1.0 + 2.0 * k * r2);
            double mu = 1.0 - (x - 1.0) / k;
            if (r3 <= 0.5 * (mu * mu + 1.0 / x)) { *ok = 1; return mu; }
        }
    }
    *ok = 0;
    return 1.0;
}

/* Waller-Hartree: a Klein-Nishina draw by Kahn's method, kept with probability
 * S(q)/Z <= 1 (the fourth word of the same block), else a new trial. */
static double or_exact_wh(double sq0, double e_kev, uint64_t seed, uint64_t h, uint32_t step, int *ok)
{
    double k = e_kev / OR_MEC2;
    double a = or_wh_a(e_kev, sq0);
    double p1 = (1.0 + 2.0 * k) / (9.0 + 2.0 * k);
    for (uint32_t t = 0; t < OR_MAX_TRIALS_WH; ++t) {
        uint32_t b[4];
        or_block(seed, h, step, OR_STREAM_EXACT | (t << 8), b);
        double r1 = or_uniform(b[0]), r2 = or_uniform(b[1]), r3 = or_uniform(b[2]), r4 = or_uniform(b[3]);
        double mu;
        if (r1 <= p1) {
            double x = 1.0 + 2.0 * k * r2;
            if (!(r3 <= 4.0 * (1.0 / x - 1.0 / (x * x)))) continue;
            mu = 1.0 - (x - 1.0) / k;
        } else {
            double x = (1.0 + 2.0 * k) / (1.0 + 2.0 * k * r2);
            mu = 1.0 - (x - 1.0) / k;
            if (!(r3 <= 0.5 * (mu * mu + 1.0 / x))) continue;
        }
        double sz = a > 0.0 ? -expm1(-a * (1.0 - mu)) : 1.0;
        if (r4 <= sz) { *ok = 1; return mu; }
    }
    *ok = 0;
    return 1.0;
}

static double or_exact_rayleigh(double q0, double e_kev, uint64_t seed, uint64_t h, uint32_t step, int *ok)
{
    double kr = e_kev / OR_HC;
    double a = q0 > 0.0 ? (2.0 * kr * kr) / (q0 * q0) : 0.0;
    for (uint32_t t = 0; t < OR_MAX_TRIALS; ++t) {
        uint32_t b[4];
        or_block(seed, h, step, OR_STREAM_EXACT | (t << 8), b);
        double z = or_uniform(b[0]), r = or_uniform(b[1]);
        double mu;
        if (a > 0.0) {
            /* 1 - mu ~ a exp(-a w) on [0, 2] */
            double w = -log1p(z * expm1(-2.0 * a)) / a;
            mu = 1.0 - w;
        } else {
            mu = 2.0 * z - 1.0;
        }
        if (mu < -1.0) mu = -1.0;
        if (r <= 0.5 * (1.0 + mu * mu)) { *ok = 1; return mu; }
    }
    *ok = 0;
    return 1.0;
}

/* Independent-atom Rayleigh: s = x^2 on [0, k^2] drawn from sum_i n_i Z_i^2 /
 * (1 + c_i s)^4 (an element with probability equal to its share of the integral,
 * then s by inverting (1 + c s)^-3), kept with probability (1 + mu^2)/2,
 * mu = 1 - 2 s / k^2.  One block per trial: element, s, acceptance. */
static double or_exact_rayleigh_iaa(const or_material *m, double e_kev, uint64_t seed, uint64_t h, uint32_t step,
                                    int *ok)
{
    double kr = e_kev / OR_HC;
    double smax = kr * kr;
    double c[OR_MAX_ELEMENTS], d[OR_MAX_ELEMENTS], w[OR_MAX_ELEMENTS];
    double total = 0.0;
    for (int i = 0; i < m->n_el; ++i) {
        double z = (double)m->el_z[i];
        c[i] = or_ff_width(m->el_z[i]);
        d[i] = -expm1(-3.0 * log1p(c[i] * smax));             /* 1 - (1 + c smax)^-3 */
        w[i] = (m->el_n[i] * (z * z)) * d[i] / (3.0 * c[i]);   /* n Z^2 int_0^smax (1 + c s)^-4 ds */
        total += w[i];
    }
    for (uint32_t t = 0; t < OR_MAX_TRIALS; ++t) {
        uint32_t b[4];
        or_block(seed, h, step, OR_STREAM_EXACT | (t << 8), b);
        double u = or_uniform(b[0]) * total, z = or_uniform(b[1]), r = or_uniform(b[2]);
        int i = 0;
        while (i < m->n_el - 1 && u >= w[i]) { u -= w[i]; ++i; }
        double s = (pow(1.0 - z * d[i], -1.0 / 3.0) - 1.0) / c[i];
        double mu = 1.0 - 2.0 * s / smax;
        if (mu < -1.0) mu = -1.0;
        if (mu > 1.0) mu = 1.0;
        if (r <= 0.5 * (1.0 + mu * mu)) { *ok = 1; return mu; }
    }
    *ok = 0;
    return 1.0;
}

/* ===================================================================== */
/* Transport in both precisions (Sec. 2.1, Fig. 2).                        */
/* ===================================================================== */
#define OR_REAL double
#define OR_SFX(n) n##_f64
#define OR_IS_F32 0
#include "ctd_oracle_transport.inc"
#undef OR_REAL
#undef OR_SFX
#undef OR_IS_F32

#define OR_REAL float
#define OR_SFX(n) n##_f32
#define OR_IS_F32 1
#include "ctd_oracle_transport.inc"
#undef OR_REAL
#undef OR_SFX
#undef OR_IS_F32
