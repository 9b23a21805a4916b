// ctd_physics.cpp -- host set-up of the transport: attenuation node tables, the
// Woodcock majorant, the R and C sampling surfaces and the stratified spectrum
// allocation.  Compiled with -ffp-contract=off: the binary64 values are rounded
// to binary32 for the device and must not depend on the host's FMA contraction.
#include <algorithm>
#include <cmath>

#include "ctd_internal.h"

namespace ctd {

// Klein-Nishina total cross section per electron in cm^2 (Eq. 2 with S = 1
// integrated over the sphere), k = E / m_e c^2.
double sigma_kn(double e_kev)
{
    const double k = e_kev / kMec2;
    const double a = 1.0 + 2.0 * k;
    const double l = std::log1p(2.0 * k);
    const double t1 = ((1.0 + k) / (k * k)) * ((2.0 * (1.0 + k)) / a - l / k);
    const double t2 = l / (2.0 * k);
    const double t3 = (1.0 + 3.0 * k) / (a * a);
    return 2.0 * kPi * kR0 * kR0 * ((t1 + t2) - t3);
}

// Incoherent scattering on free electrons: electrons per gram times sigma_KN (cm^2/g).
double mu_compton(const ctd_material &m, double e_kev)
{
    return (kNA * m.z_over_a) * sigma_kn(e_kev);
}

namespace {

// Eq. 2 up to r0^2/2: the Klein-Nishina density in mu = cos theta times the
// scattering function S/Z = 1 - exp(-a (1 - mu)), a = 2 k^2 / sq0^2 (a <= 0: 1).
inline double density_wh(double k, double a, double mu)
{
    const double e = 1.0 / (1.0 + k * (1.0 - mu));
    const double kn = (e * e) * ((e + 1.0 / e) - (1.0 - mu * mu));
    if (a <= 0.0) return kn;
    return kn * (-std::expm1(-a * (1.0 - mu)));
}

inline double wh_a(double e_kev, double sq0)
{
    const double kr = e_kev / kHc;
    return sq0 > 0.0 ? (2.0 * kr * kr) / (sq0 * sq0) : 0.0;
}

// Gauss-Legendre rule of kGaussPoints points on [-1, 1]: the roots of P_n by Newton's
// iteration from Chebyshev guesses, weights 2 / ((1 - x^2) P_n'(x)^2).
constexpr int kGaussPoints = 16;
struct GaussRule {
    double x[kGaussPoints], w[kGaussPoints];
    GaussRule()
    {
        const int n = kGaussPoints;
        for (int i = 0; i < n; ++i) {
            double z = std::cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;   // P_0, P_1, then the recurrence up to P_n
                for (int k = 2; k <= n; ++k) {
                    const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = pk;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                const double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

// Integral over mu in [-1, 1] of f(mu), the densities of Eqs. 1-2, whose features sit
// near mu = 1 (forward scattering, widths down to about 1e-3 in 1 - mu at 150 keV):
// Gauss-Legendre on panels of t = 1 - mu in [0, 2] halving toward t = 0 (2^-40 for
// the last), so that every panel is smooth at its own scale.
template <class F>
double integrate_forward(const F &f)
{
    static const GaussRule g;
    double sum = 0.0, hi = 2.0;
    for (int panel = 0; panel <= 40; ++panel) {
        const double lo = panel == 40 ? 0.0 : 0.5 * hi;
        const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
        double s = 0.0;
        for (int i = 0; i < kGaussPoints; ++i) s += g.w[i] * f(1.0 - (mid + half * g.x[i]));
        sum += half * s;
        hi = lo;
    }
    return sum;
}

}  // namespace

// Waller-Hartree total per electron in cm^2: pi r0^2 times the integral of Eq. 2
// over mu in [-1, 1] (Gauss-Legendre on panels graded toward forward scattering).
double sigma_wh(double e_kev, double sq0)
{
    const double k = e_kev / kMec2;
    const double a = wh_a(e_kev, sq0);
    return (kPi * kR0 * kR0) * integrate_forward([&](double mu) { return density_wh(k, a, mu); });
}

double mu_compton_wh(const ctd_material &m, double e_kev)
{
    return (kNA * m.z_over_a) * sigma_wh(e_kev, m.sq0);
}

namespace {

// Independent-atom form factor of Rayleigh scattering.  Each element is a screened
// hydrogenic atom: the density Z exp(-2r/a) / (pi a^3) transforms to
// F(Q) = Z / (1 + (Q a / 2)^2)^2, Q = 4 pi x, x = sin(theta/2)/lambda, with the
// Thomas-Fermi radius a = 0.8853 a0 Z^(-1/3); so F^2 = Z^2 / (1 + c x^2)^4,
// c = (2 pi a)^2.  A formula unit's F^2 is the sum over its atoms.
inline double ff_width(int z)
{
    const double a = (kThomasFermi * kBohr) / std::cbrt(static_cast<double>(z));
    const double w = (2.0 * kPi) * a;
    return w * w;
}

struct FormFactor {
    int n = 0;
    double z[CTD_MAX_ELEMENTS], count[CTD_MAX_ELEMENTS], c[CTD_MAX_ELEMENTS];
    explicit FormFactor(const Elements &el) : n(el.n)
    {
        for (int i = 0; i < n; ++i) {
            z[i] = static_cast<double>(el.z[i]);
            count[i] = el.count[i];
            c[i] = ff_width(el.z[i]);
        }
    }
    // F^2 of the formula unit at x^2
    double f2(double x2) const
    {
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            const double g = 1.0 / (1.0 + c[i] * x2);
            const double f = z[i] * (g * g);
            s += count[i] * (f * f);
        }
        return s;
    }
    // Eq. 1 up to r0^2/2 at polar cosine mu, kr = E/hc: (1 + mu^2) F^2, x^2 = kr^2 (1 - mu) / 2
    double density(double kr, double mu) const
    {
        const double x2 = ((kr * kr) * (1.0 - mu)) * 0.5;
        return (1.0 + mu * mu) * f2(x2);
    }
};

}  // namespace

// Rayleigh total per formula unit in cm^2 with the independent-atom form factor:
// pi r0^2 times the integral of Eq. 1 over mu in [-1, 1] (Gauss-Legendre on panels
// graded toward forward scattering).
double sigma_rayleigh_iaa(const Elements &el, double e_kev)
{
    const FormFactor ff(el);
    const double kr = e_kev / kHc;
    return (kPi * kR0 * kR0) * integrate_forward([&](double mu) { return ff.density(kr, mu); });
}

double mu_rayleigh_iaa(const ctd_material &m, const Elements &el, double e_kev)
{
    return (sigma_rayleigh_iaa(el, e_kev) * kNA) / m.a_mol;
}

// Photoelectric absorption, 1e-2 Z^4 / E_MeV^3 microbarn per formula unit (cm^2/g).
double mu_pe(const ctd_material &m, double e_kev)
{
    const double em = e_kev / 1000.0;
    const double z2 = m.z_eff * m.z_eff;
    const double sigma = kPeCoef * (z2 * z2) / (em * em * em);
    return ((sigma * kMicrobarn) * kNA) / m.a_mol;
}

// Rayleigh scattering, 1.565e-5 Z^2 / E_MeV^2 barn per formula unit (cm^2/g).
double mu_rayleigh(const ctd_material &m, double e_kev)
{
    const double em = e_kev / 1000.0;
    const double z2 = m.z_eff * m.z_eff;
    const double sigma = kRayCoef * z2 / (em * em);
    return ((sigma * kBarn) * kNA) / m.a_mol;
}

void material_columns(const ctd_material &mat, const Elements &el, int e_min, int n_e, int compton_model,
                      double *out)
{
    for (int j = 0; j < n_e; ++j) {
        const double e = static_cast<double>(e_min + j);
        const double pe = mu_pe(mat, e);
        const double c = compton_model == CTD_COMPTON_WH ? mu_compton_wh(mat, e) : mu_compton(mat, e);
        const double r = el.n > 0 ? mu_rayleigh_iaa(mat, el, e) : mu_rayleigh(mat, e);
        double *dst = out + static_cast<size_t>(j) * 3;
        dst[0] = pe;
        dst[1] = pe + c;
        dst[2] = (pe + c) + r;
    }
}

void build_majorant(const std::vector<double> &cum, const std::vector<double> &rho_max, const std::vector<int> &present,
                    int n_e, double scale, std::vector<double> &mmax)
{
    const size_t nm = rho_max.size();
    mmax.assign(n_e, 0.0);
    // mu_max(E): the largest total attenuation anywhere in the volume
    for (int j = 0; j < n_e; ++j) {
        double best = 0.0;
        for (size_t m = 0; m < nm; ++m) {
            if (!present[m]) continue;
            const double v = rho_max[m] * cum[(m * n_e + j) * 3 + 2];
            if (v > best) best = v;
        }
        mmax[j] = scale * best;
    }
}

namespace {

// unnormalised polar-cosine densities of Eq. 2 (S = 1) and Eq. 1 with F^2 = exp(-q^2/q0^2)
inline double density_kn(double k, double mu)
{
    const double e = 1.0 / (1.0 + k * (1.0 - mu));
    return (e * e) * ((e + 1.0 / e) - (1.0 - mu * mu));
}

inline double density_rayleigh(double a, double mu)
{
    if (a <= 0.0) return 1.0 + mu * mu;
    return (1.0 + mu * mu) * std::exp(-a * (1.0 - mu));
}

inline double grid_mu(int n)
{
    return static_cast<double>(2 * n - kCdfIntervals) / static_cast<double>(kCdfIntervals);
}

}  // namespace

void build_surface(int kind, double q0, const Elements *el, int e_min, int n_e, int n_zeta, double *out)
{
    const int M = kCdfIntervals;
    std::vector<double> pdf(M + 1), cdf(M + 1);
    const FormFactor ff(kind == 3 && el ? *el : Elements{});
    for (int j = 0; j < n_e; ++j) {
        const double e = static_cast<double>(e_min + j);
        const double k = e / kMec2;
        const double kr = e / kHc;
        const double a = q0 > 0.0 ? (2.0 * kr * kr) / (q0 * q0) : 0.0;
        for (int n = 0; n <= M; ++n)
            pdf[n] = kind == 0   ? density_kn(k, grid_mu(n))
                     : kind == 1 ? density_rayleigh(a, grid_mu(n))
                     : kind == 2 ? density_wh(k, a, grid_mu(n))
                                 : ff.density(kr, grid_mu(n));
        // cumulative trapezoid without the common factor h/2
        cdf[0] = 0.0;
        for (int n = 1; n <= M; ++n) cdf[n] = cdf[n - 1] + (pdf[n - 1] + pdf[n]);
        double *row = out + static_cast<size_t>(j) * n_zeta;
        const double total = cdf[M];
        int n = 0;
        row[0] = -1.0;
        for (int i = 1; i < n_zeta - 1; ++i) {
            const double target = (static_cast<double>(i) / static_cast<double>(n_zeta - 1)) * total;
            while (n < M - 1 && cdf[n + 1] <= target) ++n;
            const double m0 = grid_mu(n), m1 = grid_mu(n + 1);
            row[i] = m0 + ((target - cdf[n]) / (cdf[n + 1] - cdf[n])) * (m1 - m0);
        }
        row[n_zeta - 1] = 1.0;
    }
}

bool alias_build(int n, const double *f, uint32_t *thr, int32_t *alias)
{
    if (n <= 0) return false;
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(f[i] >= 0.0) || !std::isfinite(f[i])) return false;
        total += f[i];
    }
    if (!(total > 0.0) || !std::isfinite(total)) return false;
    // n f_i / total: columns under 1 are filled up from columns over 1, taken
    // last in, first out from two work lists
    std::vector<double> p(n);
    std::vector<int> under, over;
    under.reserve(n);
    over.reserve(n);
    for (int i = 0; i < n; ++i) {
        p[i] = (f[i] * static_cast<double>(n)) / total;
        if (p[i] < 1.0) under.push_back(i);
        else over.push_back(i);
    }
    while (!under.empty() && !over.empty()) {
        const int l = under.back(), g = over.back();
        under.pop_back();
        over.pop_back();
        thr[l] = static_cast<uint32_t>(p[l] * 4294967296.0);
        alias[l] = g;
        p[g] = (p[g] + p[l]) - 1.0;
        if (p[g] < 1.0) under.push_back(g);
        else over.push_back(g);
    }
    // columns left over hold 1 up to rounding
    while (!over.empty()) {
        const int g = over.back();
        over.pop_back();
        thr[g] = 0xffffffffu;
        alias[g] = g;
    }
    while (!under.empty()) {
        const int l = under.back();
        under.pop_back();
        thr[l] = 0xffffffffu;
        alias[l] = l;
    }
    return true;
}

bool allocate(uint64_t n, const std::vector<double> &w, std::vector<uint64_t> &out)
{
    // Largest remainder (Sec. 2.2.5): quota n w_j / W, its floor to every bin, then one
    // more to the bins of largest fractional part (ties to the lower bin, none to
    // empty bins) until the counts add up to n.  Weights must be finite, >= 0, and
    // sum to a finite positive W.
    const size_t nb = w.size();
    if (nb == 0) return false;
    double total = 0.0;
    for (double x : w) {
        if (!(x >= 0.0) || !std::isfinite(x)) return false;
        total += x;
    }
    if (!(total > 0.0) || !std::isfinite(total)) return false;
    out.assign(nb, 0);
    std::vector<double> frac(nb);
    uint64_t given = 0;
    for (size_t j = 0; j < nb; ++j) {
        const double q = static_cast<double>(n) * w[j] / total;
        const double f = std::floor(q);
        out[j] = static_cast<uint64_t>(f);
        frac[j] = q - f;
        given += out[j];
    }
    if (given < n) {
        // bins of positive weight by decreasing fraction, lower bin first among equals
        std::vector<size_t> order;
        for (size_t j = 0; j < nb; ++j)
            if (w[j] > 0.0) order.push_back(j);
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return frac[a] > frac[b]; });
        for (size_t i = 0; i < order.size() && given < n; ++i, ++given) ++out[order[i]];
        // rounding of the quotas could in principle leave more than one per bin: the
        // rest goes to the lowest bin of positive weight
        if (given < n) {
            out[order.front()] += n - given;
            given = n;
        }
    } else if (given > n) {
        // rounding pushed the floors past n: one back from each bin of smallest
        // fraction among those holding any, the higher bin first among equals
        std::vector<size_t> order;
        for (size_t j = nb; j-- > 0;)
            if (out[j] > 0) order.push_back(j);
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return frac[a] < frac[b]; });
        for (size_t i = 0; i < order.size() && given > n; ++i, --given) --out[order[i]];
    }
    return given == n;
}

}  // namespace ctd
