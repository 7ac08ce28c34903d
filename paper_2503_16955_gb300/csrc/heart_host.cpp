// heart_host.cpp -- per-spectrometer set-up on the host: descriptor
// validation, frames, rocking-curve constants and the mosaic inverse-CDF table
// that the kernels stage in shared memory.  Runs once per heart_spectrometer_create;
// no ray is traced here.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "heart_internal.h"

namespace heart {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kHcKeVA = 12.398419843320026;   // h c, keV Angstrom

int set_err(char *err, int n, const char *m) {
    std::snprintf(err, (size_t)n, "%s", m);
    return 1;
}

double dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
void cross(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
bool unit(const double *in, double *out) {
    double n = std::sqrt(dot(in, in));
    if (!(n > 0) || !std::isfinite(n)) return false;
    for (int i = 0; i < 3; ++i) out[i] = in[i] / n;
    return true;
}
// component of a perpendicular to the unit vector n, normalised
bool perp_unit(const double *a, const double *n, double *out) {
    double d = dot(a, n), t[3];
    for (int i = 0; i < 3; ++i) t[i] = a[i] - d * n[i];
    double len = std::sqrt(dot(t, t));
    if (!(len > 1e-12 * std::sqrt(dot(a, a)))) return false;
    for (int i = 0; i < 3; ++i) out[i] = t[i] / len;
    return true;
}
bool finite3(const double *a) { return std::isfinite(a[0]) && std::isfinite(a[1]) && std::isfinite(a[2]); }

// ---------------------------------------------------------------------------
// 5-point Gauss-Legendre rule (nodes and weights in closed form)
// ---------------------------------------------------------------------------
struct GL5 {
    double x[5], w[5];
    GL5() {
        double a = std::sqrt(5.0 - 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
        double b = std::sqrt(5.0 + 2.0 * std::sqrt(10.0 / 7.0)) / 3.0;
        double wa = (322.0 + 13.0 * std::sqrt(70.0)) / 900.0;
        double wb = (322.0 - 13.0 * std::sqrt(70.0)) / 900.0;
        double xs[5] = {-b, -a, 0.0, a, b}, ws[5] = {wb, wa, 128.0 / 225.0, wa, wb};
        for (int i = 0; i < 5; ++i) { x[i] = xs[i]; w[i] = ws[i]; }
    }
    template <class F> double operator()(const F &f, double lo, double hi) const {
        double m = 0.5 * (lo + hi), h = 0.5 * (hi - lo), s = 0.0;
        for (int i = 0; i < 5; ++i) s += w[i] * f(m + h * x[i]);
        return s * h;
    }
};

// ---------------------------------------------------------------------------
// mosaic distribution: the quantity tabulated is q = 1 - cos(theta), whose
// density on the sphere is proportional to W (dq = sin(theta) dtheta)
// ---------------------------------------------------------------------------
struct MdfShape {
    int kind;
    double G, eta;
    // W as a function of theta, for the shapes defined in theta
    double W(double th) const {
        const double c = 4.0 * kLn2 / (G * G);
        switch (kind) {
        case HEART_MDF_GAUSSIAN: return std::exp(-c * th * th);
        case HEART_MDF_LORENTZIAN: return 1.0 / (0.25 * G * G + th * th);
        case HEART_MDF_PSEUDO_VOIGT: {
            double L = (G / (2.0 * kPi)) / (0.25 * G * G + th * th);
            double Gs = std::sqrt(c / kPi) * std::exp(-c * th * th);
            return eta * L + (1.0 - eta) * Gs;
        }
        }
        return 0.0;
    }
};

// Numerical inverse CDF for the theta-defined shapes: cell integrals of
// W(theta) sin(theta) on a geometric theta grid, cumulated from both ends,
// then Newton inside the cell that holds the target mass.
class NumericMdf {
  public:
    explicit NumericMdf(const MdfShape &s) : s_(s) {
        const double first = 1e-7 * s.G, ratio = 1.002;
        th_.push_back(0.0);
        for (double t = first; t < kPi; t *= ratio) th_.push_back(t);
        th_.push_back(kPi);
        size_t n = th_.size() - 1;
        cell_.resize(n);
        for (size_t i = 0; i < n; ++i) cell_[i] = gl_(f_, th_[i], th_[i + 1]);
        lo_.assign(n + 1, 0.0L);
        hi_.assign(n + 1, 0.0L);
        for (size_t i = 0; i < n; ++i) lo_[i + 1] = lo_[i] + cell_[i];
        for (size_t i = n; i-- > 0;) hi_[i] = hi_[i + 1] + cell_[i];
        total_ = (double)hi_[0];
    }
    double total() const { return total_; }
    // theta with F(theta) = u (from_top = false) or 1 - F(theta) = c (true)
    double theta_at(double frac, bool from_top) const {
        const size_t n = cell_.size();
        long double target = (long double)frac * (long double)total_;
        size_t j;
        long double rem;
        if (!from_top) {
            size_t a = 0, b = n;        // largest j with lo_[j] <= target
            while (b - a > 1) { size_t m = (a + b) / 2; if (lo_[m] <= target) a = m; else b = m; }
            j = a;
            rem = target - lo_[j];
        } else {
            size_t a = 0, b = n;        // largest j with hi_[j] > target
            while (b - a > 1) { size_t m = (a + b) / 2; if (hi_[m] > target) a = m; else b = m; }
            j = a;
            rem = target - hi_[j + 1];
        }
        double t0 = th_[j], t1 = th_[j + 1], c = cell_[j];
        double r = (double)rem;
        if (!(c > 0)) return from_top ? t0 : t1;
        double lo = t0, hi = t1;
        double t = from_top ? t1 - (t1 - t0) * (r / c) : t0 + (t1 - t0) * (r / c);
        for (int it = 0; it < 60; ++it) {
            double g = from_top ? gl_(f_, t, t1) - r : gl_(f_, t0, t) - r;
            bool left = from_top ? (g > 0) : (g < 0);
            if (left) lo = t; else hi = t;
            double d = f_(t);
            double tn = (d > 0) ? (from_top ? t + g / d : t - g / d) : 0.5 * (lo + hi);
            if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
            if (std::fabs(tn - t) <= 2e-16 * t || hi - lo <= 2e-16 * hi) { t = tn; break; }
            t = tn;
        }
        return t;
    }

  private:
    struct Fn {
        const MdfShape *s;
        double operator()(double th) const { return s->W(th) * std::sin(th); }
    };
    MdfShape s_;
    Fn f_{&s_};
    GL5 gl_;
    std::vector<double> th_, cell_;
    std::vector<long double> lo_, hi_;
    double total_ = 0.0;
};

double q_of_theta(double th) {
    double h = std::sin(0.5 * th);
    return 2.0 * h * h;
}

// closed-form quantiles of q for the shapes defined in q; `comp` = 1 - u
double closed_form_q(int kind, double G, double u, double comp) {
    switch (kind) {
    case HEART_MDF_VMF: {          // density exp(-q / s^2) on [0, 2]
        double s2 = G * G / (8.0 * kLn2);
        double m = -std::expm1(-2.0 / s2);            // 1 - exp(-2/s^2)
        if (comp < 0.5) return -s2 * std::log(comp * m + std::exp(-2.0 / s2));
        return -s2 * std::log1p(-u * m);
    }
    case HEART_MDF_WRAPPED_LORENTZIAN: {   // density 1 / (a^2 + 2q)
        double a2 = 0.25 * G * G;
        return 0.5 * a2 * std::expm1(u * std::log1p(4.0 / a2));
    }
    case HEART_MDF_SPHERICAL_WRAPPED_LORENTZIAN: {  // density 1 / (b + q)^2
        double sh = std::sinh(0.25 * G), b = 2.0 * sh * sh;
        double inv = (comp < 0.5) ? 1.0 / (b + 2.0) + comp * (1.0 / b - 1.0 / (b + 2.0))
                                  : 1.0 / b - u * (1.0 / b - 1.0 / (b + 2.0));
        return 1.0 / inv - b;
    }
    case HEART_MDF_UNIFORM: {
        double h = std::sin(0.25 * G);
        return u * 2.0 * h * h;
    }
    }
    return 0.0;
}

// table: knots [0, kMdfM) at u = i / kMdfM, then kMdfT + 1 tail knots at
// 1 - u = 2^-tau, tau = 12 + 21 j / kMdfT
int build_mdf_table(const heart_spectrometer_desc *d, double *tab) {
    int kind = d->mdf;
    double G = d->mdf_fwhm_rad;
    if (kind == HEART_MDF_GAUSSIAN || kind == HEART_MDF_LORENTZIAN || kind == HEART_MDF_PSEUDO_VOIGT) {
        MdfShape s{kind, G, d->mdf_eta};
        NumericMdf nm(s);
        if (!(nm.total() > 0)) return 1;
        tab[0] = 0.0;
        for (int i = 1; i < kMdfM; ++i) tab[i] = q_of_theta(nm.theta_at((double)i / kMdfM, false));
        for (int j = 0; j <= kMdfT; ++j) {
            double tau = 12.0 + 21.0 * (double)j / kMdfT;
            tab[kMdfM + j] = q_of_theta(nm.theta_at(std::exp2(-tau), true));
        }
    } else {
        tab[0] = 0.0;
        for (int i = 1; i < kMdfM; ++i) {
            double u = (double)i / kMdfM;
            tab[i] = closed_form_q(kind, G, u, 1.0 - u);
        }
        for (int j = 0; j <= kMdfT; ++j) {
            double c = std::exp2(-(12.0 + 21.0 * (double)j / kMdfT));
            tab[kMdfM + j] = closed_form_q(kind, G, 1.0 - c, c);
        }
    }
    tab[kMdfM - 1] = tab[kMdfM];   // the body's last knot is the tail's first (u = 1 - 1/M)
    for (int i = 0; i < kMdfKnots; ++i)
        if (!std::isfinite(tab[i])) return 1;
    return 0;
}

// ---------------------------------------------------------------------------
// rocking curves
// ---------------------------------------------------------------------------
void pseudo_voigt(double fg, double fl, double *F, double *eta) {
    // total width (fifth-order polynomial) and mixing (cubic), Sec. 2.2.1
    double g2 = fg * fg, g3 = g2 * fg, g4 = g3 * fg, g5 = g4 * fg;
    double l2 = fl * fl, l3 = l2 * fl, l4 = l3 * fl, l5 = l4 * fl;
    double s = g5 + 2.69269 * g4 * fl + 2.42843 * g3 * l2 + 4.47163 * g2 * l3 + 0.07842 * fg * l4 + l5;
    *F = std::pow(s, 0.2);
    double r = fl / *F;
    *eta = ((0.11116 * r - 0.47719) * r + 1.36603) * r;
}

double dp_reflectivity(double y, double g) {
    // |eta - sqrt(eta^2 - 1)|^2 with eta = y + i g, written as 1 / max(|eta -+ z|)^2
    double ar = y * y - g * g - 1.0, ai = 2.0 * y * g;     // eta^2 - 1
    double r = std::hypot(ar, ai);
    double zr, zi;
    if (ar >= 0) { zr = std::sqrt(0.5 * (r + ar)); zi = (zr > 0) ? 0.5 * ai / zr : 0.0; }
    else { zi = std::copysign(std::sqrt(0.5 * (r - ar)), ai); zr = 0.5 * ai / zi; }
    double m1 = std::hypot(y - zr, g - zi), m2 = std::hypot(y + zr, g + zi);
    double m = m1 > m2 ? m1 : m2;
    return 1.0 / (m * m);
}

double dp_area(double g) {
    // 2 * int_0^inf R dy with y = tan(phi): integrand R(tan phi) sec^2(phi)
    GL5 gl;
    auto f = [g](double phi) {
        double y = std::tan(phi);
        if (!(y < 1e150)) return 0.25;
        return dp_reflectivity(y, g) * (1.0 + y * y);
    };
    const int n = 4096;
    long double s = 0.0L;
    for (int half = 0; half < 2; ++half) {
        double a = half ? 0.25 * kPi : 0.0, b = half ? 0.5 * kPi : 0.25 * kPi;
        for (int i = 0; i < n; ++i) s += gl(f, a + (b - a) * i / n, a + (b - a) * (i + 1) / n);
    }
    return 2.0 * (double)s;
}

// W(q) / W(0) of the mosaic distribution in closed form, and for a spectrometer
// without rocking curve the cone-candidate factor 2 W(0) / int_0^qmax W dq
// (2 cones x 2 pi f(0), f = W / (2 pi int W dq) per unit solid angle)
void mdf_ratio_params(const heart_spectrometer_desc *d, SpecParams *p) {
    const double G = d->mdf_fwhm_rad;
    p->mdf = d->mdf;
    p->w_a2 = 0.25 * G * G;
    double W0 = 1.0, norm = 0.0;
    switch (d->mdf) {
    case HEART_MDF_GAUSSIAN:
    case HEART_MDF_LORENTZIAN:
    case HEART_MDF_PSEUDO_VOIGT: {
        const double c = 4.0 * kLn2 / (G * G);
        p->w_c = c;
        const MdfShape sh{d->mdf, G, d->mdf_eta};
        W0 = sh.W(0.0);
        if (d->mdf == HEART_MDF_GAUSSIAN) { p->w_wl = 0.0; p->w_wg = 1.0; }
        else if (d->mdf == HEART_MDF_LORENTZIAN) { p->w_wl = 1.0; p->w_wg = 0.0; }
        else {
            p->w_wl = d->mdf_eta * (2.0 / (kPi * G)) / W0;
            p->w_wg = (1.0 - d->mdf_eta) * std::sqrt(c / kPi) / W0;
        }
        if (d->irc == HEART_IRC_NONE) norm = NumericMdf(sh).total();
        break;
    }
    case HEART_MDF_VMF: {
        const double s2 = G * G / (8.0 * kLn2);
        p->w_c = 1.0 / s2;
        norm = -s2 * std::expm1(-2.0 / s2);
        break;
    }
    case HEART_MDF_WRAPPED_LORENTZIAN:
        W0 = 1.0 / p->w_a2;
        norm = 0.5 * std::log1p(4.0 / p->w_a2);
        break;
    case HEART_MDF_SPHERICAL_WRAPPED_LORENTZIAN: {
        const double sh = std::sinh(0.25 * G);
        p->w_b = 2.0 * sh * sh;
        W0 = 1.0 / (p->w_b * p->w_b);
        norm = 1.0 / p->w_b - 1.0 / (p->w_b + 2.0);
        break;
    }
    default: {
        const double h = std::sin(0.25 * G);
        p->w_qmax = 2.0 * h * h;
        norm = p->w_qmax;
        break;
    }
    }
    p->none_fac = (d->irc == HEART_IRC_NONE && norm > 0) ? 2.0 * W0 / norm : 0.0;
}

// W(q) / W(0) from the closed-form parameters above (as the kernels evaluate it)
double mdf_ratio_host(const SpecParams &p, double q) {
    switch (p.mdf) {
    case HEART_MDF_VMF: return std::exp(-p.w_c * q);
    case HEART_MDF_WRAPPED_LORENTZIAN: return p.w_a2 / (p.w_a2 + 2.0 * q);
    case HEART_MDF_SPHERICAL_WRAPPED_LORENTZIAN: {
        const double r = p.w_b / (p.w_b + q);
        return r * r;
    }
    case HEART_MDF_UNIFORM: return q <= p.w_qmax ? 1.0 : 0.0;
    default: {
        const double th = 2.0 * std::asin(std::sqrt(0.5 * std::fmin(std::fmax(q, 0.0), 2.0)));
        return p.w_wl * (p.w_a2 / (p.w_a2 + th * th)) + p.w_wg * std::exp(-p.w_c * th * th);
    }
    }
}

// the cone sampler's window tilt q_v: W(q) / W(0) <= v* for every q >= q_v (the
// mosaic distributions decrease with the tilt); 100 bisection steps on [0, 2],
// widened by 1e-9 relative; infinite if W(2) / W(0) > v*
double none_window_tilt(const SpecParams &p) {
    if (mdf_ratio_host(p, 2.0) > p.vstar) return INFINITY;
    double lo = 0.0, hi = 2.0;
    for (int i = 0; i < 100; ++i) {
        const double m = 0.5 * (lo + hi);
        if (mdf_ratio_host(p, m) <= p.vstar) hi = m; else lo = m;
    }
    return hi * (1.0 + 1e-9);
}

}  // namespace

heart_status build_spec_params(const heart_spectrometer_desc *d, SpecParams *p, double *tab,
                               char *err, int errlen) {
    std::memset(p, 0, sizeof *p);
#define REQUIRE(cond, msg) do { if (!(cond)) { set_err(err, errlen, msg); return HEART_EINVAL; } } while (0)
    REQUIRE(d, "null spectrometer descriptor");
    REQUIRE(d->d_spacing_A > 0 && std::isfinite(d->d_spacing_A), "d_spacing_A must be > 0");
    REQUIRE(d->thickness_mm > 0 && std::isfinite(d->thickness_mm), "thickness_mm must be > 0");
    REQUIRE(d->size_disp_mm > 0 && d->size_nondisp_mm > 0, "crystal sizes must be > 0");
    REQUIRE(d->geometry == HEART_FLAT || d->geometry == HEART_CYL_VON_HAMOS, "unknown geometry");
    REQUIRE(d->mdf >= HEART_MDF_GAUSSIAN && d->mdf <= HEART_MDF_UNIFORM, "unknown mdf");
    REQUIRE(d->mdf_fwhm_rad > 0 && d->mdf_fwhm_rad < 1.0, "mdf_fwhm_rad must be in (0, 1) rad");
    REQUIRE(d->mdf != HEART_MDF_PSEUDO_VOIGT || (d->mdf_eta >= 0 && d->mdf_eta <= 1), "mdf_eta in [0,1]");
    REQUIRE(d->irc >= HEART_IRC_DARWIN && d->irc <= HEART_IRC_NONE, "unknown irc");
    REQUIRE(d->irc == HEART_IRC_NONE || (d->irc_fwhm_rad > 0 && d->irc_fwhm_rad < 0.1),
            "irc_fwhm_rad must be in (0, 0.1) rad");
    REQUIRE(d->irc != HEART_IRC_PSEUDO_VOIGT || d->irc_lorentz_fwhm_rad >= 0, "irc_lorentz_fwhm_rad >= 0");
    REQUIRE(d->irc != HEART_IRC_DARWIN_PRINS || d->prins_g >= 0, "prins_g >= 0");
    REQUIRE(std::isfinite(d->irc_shift_rad) && std::fabs(d->irc_shift_rad) < 0.1, "irc_shift_rad");
    REQUIRE(d->absorption_length_mm > 0 && d->absorption_ref_keV > 0 && std::isfinite(d->absorption_power),
            "absorption length / reference energy must be > 0");
    REQUIRE(d->refl_K_per_mm2 >= 0 || (d->refl_darwin_fwhm_rad > 0 && d->refl_ref_keV > 0),
            "K < 0 needs refl_darwin_fwhm_rad > 0 and refl_ref_keV > 0");
    REQUIRE(d->max_reflections >= 0 && d->max_reflections <= 1000000, "max_reflections in [0, 1e6]");
    REQUIRE(d->max_collisions >= 1, "max_collisions >= 1");
    REQUIRE(d->det_nx >= 1 && d->det_ny >= 1 && d->det_nx <= 65536 && d->det_ny <= 65536, "detector size");
    REQUIRE(d->pixel_mm > 0 && std::isfinite(d->pixel_mm), "pixel_mm must be > 0");
    REQUIRE(d->count_type == HEART_COUNT_I32 || d->count_type == HEART_COUNT_I64, "count_type");
    REQUIRE(finite3(d->centre_mm) && finite3(d->det_centre_mm), "non-finite position");

    p->geometry = d->geometry;
    p->irc = d->irc;
    p->max_refl = d->max_reflections;
    p->count_type = d->count_type;
    REQUIRE(d->sampler == HEART_SAMPLER_THINNED || d->sampler == HEART_SAMPLER_PLAIN, "sampler");
    REQUIRE(d->thin_vstar >= 0 && d->thin_vstar < 1, "thin_vstar in [0, 1)");
    p->sampler = d->sampler;
    p->vstar = d->thin_vstar > 0 ? d->thin_vstar : 1.0 / 64.0;     // X* is set by the caller
    REQUIRE(d->n_orders >= 0 && d->n_orders <= HEART_MAX_ORDERS, "0..4 reflection orders");
    p->n_orders = d->n_orders > 0 ? d->n_orders : 1;
    if (d->n_orders == 0) {
        p->ord_m[0] = 1;
        p->ord_k[0] = 1.0;
        p->ord_w[0] = 1.0;
    }
    for (int h = 0; h < d->n_orders; ++h) {
        REQUIRE(d->order_m[h] >= 1 && std::isfinite(d->order_K_rel[h]) && d->order_K_rel[h] >= 0 &&
                    std::isfinite(d->order_w_rel[h]) && d->order_w_rel[h] > 0,
                "order: multiple >= 1, K ratio >= 0, width ratio > 0");
        p->ord_m[h] = d->order_m[h];
        p->ord_k[h] = d->order_K_rel[h];
        p->ord_w[h] = d->order_w_rel[h];
    }
    REQUIRE(d->n_irc_e >= 0 && d->n_irc_e <= HEART_MAX_IRC_E, "0..16 energy knots of the rocking curve");
    p->n_irc_e = d->n_irc_e;
    for (int i = 0; i < d->n_irc_e; ++i) {
        REQUIRE(std::isfinite(d->irc_e_wscale[i]) && d->irc_e_wscale[i] > 0 && std::isfinite(d->irc_e_shift_rad[i]),
                "rocking-curve energy knots: width scale > 0, finite shift");
        if (i > 0) REQUIRE(d->irc_e_keV[i] > d->irc_e_keV[i - 1], "rocking-curve energy knots must ascend");
        p->irc_e[i] = d->irc_e_keV[i];
        p->irc_ws[i] = d->irc_e_wscale[i];
        p->irc_sh[i] = d->irc_e_shift_rad[i];
    }
    p->max_coll = d->max_collisions;
    p->thickness = d->thickness_mm;
    p->radius = d->radius_mm;
    for (int i = 0; i < 3; ++i) p->c[i] = d->centre_mm[i];
    if (d->geometry == HEART_FLAT) {
        REQUIRE(unit(d->normal, p->N), "bad normal");
        REQUIRE(perp_unit(d->axis, p->N, p->ed), "axis parallel to the normal");
        cross(p->N, p->ed, p->en);
        p->half_d = 0.5 * d->size_disp_mm;
        p->half_n = 0.5 * d->size_nondisp_mm;
    } else {
        REQUIRE(d->radius_mm > 0 && std::isfinite(d->radius_mm), "radius_mm must be > 0");
        REQUIRE(unit(d->axis, p->ax), "bad axis");
        REQUIRE(perp_unit(d->normal, p->ax, p->cc), "normal parallel to the axis");
        cross(p->ax, p->cc, p->ww);
        double half = 0.5 * d->size_nondisp_mm / d->radius_mm;
        REQUIRE(half < 0.5 * kPi, "arc length must be below pi R");
        p->sphi = std::sin(half);
        p->cphi = std::cos(half);
        p->zc = d->centre_axial_mm;
        p->half_d = 0.5 * d->size_disp_mm;
        REQUIRE(std::isfinite(p->zc), "centre_axial_mm");
    }
    REQUIRE(unit(d->det_u, p->eu), "bad det_u");
    REQUIRE(perp_unit(d->det_v, p->eu, p->ev), "det_v parallel to det_u");
    cross(p->eu, p->ev, p->nd);
    for (int i = 0; i < 3; ++i) p->D0[i] = d->det_centre_mm[i];
    p->nx = d->det_nx;
    p->ny = d->det_ny;
    p->pix = d->pixel_mm;

    // rocking curve
    p->irc_shift = d->irc_shift_rad;
    p->irc_fwhm = d->irc_fwhm_rad;
    p->irc_delta = d->irc_fwhm_rad * std::sqrt(2.0) / 3.0;
    p->irc_g = d->prins_g;
    switch (d->irc) {
    case HEART_IRC_DARWIN:
        p->irc_norm = p->irc_delta * 8.0 / 3.0;
        p->irc_max = 1.0 / p->irc_norm;
        break;
    case HEART_IRC_DARWIN_PRINS: {
        p->irc_norm = p->irc_delta * dp_area(d->prins_g);
        double m = 0.0;
        for (int i = 0; i <= 8000; ++i) {            // the curve peaks at y = 0; scan to be sure
            double r = dp_reflectivity(-4.0 + 8.0 * i / 8000, d->prins_g);
            if (r > m) m = r;
        }
        p->irc_max = m / p->irc_norm;
        break;
    }
    case HEART_IRC_PSEUDO_VOIGT:
        pseudo_voigt(d->irc_fwhm_rad, d->irc_lorentz_fwhm_rad, &p->irc_fwhm, &p->irc_eta);
        p->irc_max = p->irc_eta * 2.0 / (kPi * p->irc_fwhm) +
                     (1.0 - p->irc_eta) * std::sqrt(4.0 * kLn2 / kPi) / p->irc_fwhm;
        break;
    case HEART_IRC_GAUSSIAN: p->irc_max = std::sqrt(4.0 * kLn2 / kPi) / p->irc_fwhm; break;
    case HEART_IRC_LORENTZIAN: p->irc_max = 2.0 / (kPi * p->irc_fwhm); break;
    case HEART_IRC_BOX: p->irc_max = 1.0 / p->irc_fwhm; break;
    case HEART_IRC_NONE: p->irc_max = 0.0; break;    // a delta function: the cone candidates take over
    }
    mdf_ratio_params(d, p);
    p->none_qv = d->irc == HEART_IRC_NONE ? none_window_tilt(*p) : INFINITY;

    // physics
    p->d_A = d->d_spacing_A;
    p->labs = d->absorption_length_mm;
    p->labs_ref = d->absorption_ref_keV;
    p->labs_pow = d->absorption_power;
    if (d->refl_K_per_mm2 >= 0) {
        p->K = d->refl_K_per_mm2;
    } else {
        // Darwin half-width delta = K lambda^2 / (pi sin 2 aB) at the reference energy
        double lam_A = kHcKeVA / d->refl_ref_keV;
        double sb = lam_A / (2.0 * d->d_spacing_A);
        REQUIRE(sb < 1.0, "no Bragg reflection at refl_ref_keV");
        double cb = std::sqrt(1.0 - sb * sb), lam = lam_A * 1e-7;
        double delta = d->refl_darwin_fwhm_rad * std::sqrt(2.0) / 3.0;
        p->K = kPi * delta * 2.0 * sb * cb / (lam * lam);
    }
    if (build_mdf_table(d, tab)) { set_err(err, errlen, "mosaic table construction failed"); return HEART_EINVAL; }
#undef REQUIRE
    return HEART_OK;
}

heart_status build_source_params(const heart_source_desc *s, SourceParams *p, char *err, int errlen,
                                 std::vector<unsigned char> *spectrum) {
    std::memset(p, 0, sizeof *p);
    if (spectrum) spectrum->clear();
#define REQUIRE(cond, msg) do { if (!(cond)) { set_err(err, errlen, msg); return HEART_EINVAL; } } while (0)
    REQUIRE(s, "null source descriptor");
    REQUIRE(s->components && s->n_components >= 1 && s->n_components <= kMaxComp, "1..16 components");
    REQUIRE(s->cone_half_angle_rad >= 0 && s->cone_half_angle_rad <= kPi, "cone half-angle in [0, pi]");
    REQUIRE(s->spot_fwhm_mm[0] >= 0 && s->spot_fwhm_mm[1] >= 0, "spot FWHM >= 0");
    REQUIRE(finite3(s->origin_mm), "non-finite origin");
    double tot = 0.0;
    for (int i = 0; i < s->n_components; ++i) {
        const heart_spectral_component &c = s->components[i];
        REQUIRE(c.weight >= 0 && std::isfinite(c.weight), "component weight >= 0");
        REQUIRE(c.kind >= HEART_SRC_MONO && c.kind <= HEART_SRC_TABLE, "unknown component kind");
        if (c.kind == HEART_SRC_MONO || c.kind == HEART_SRC_GAUSS || c.kind == HEART_SRC_LORENTZ)
            REQUIRE(c.e0_keV > 0 && std::isfinite(c.e0_keV), "e0_keV must be > 0");
        if (c.kind == HEART_SRC_GAUSS) REQUIRE(c.width_keV >= 0, "Gaussian sigma >= 0");
        if (c.kind == HEART_SRC_LORENTZ) REQUIRE(c.width_keV > 0, "Lorentzian FWHM > 0");
        if (c.kind == HEART_SRC_INV_E) REQUIRE(c.lo_keV > 0 && c.hi_keV > c.lo_keV, "1/E needs 0 < lo < hi");
        if (c.kind == HEART_SRC_UNIFORM) REQUIRE(c.lo_keV > 0 && c.hi_keV >= c.lo_keV, "uniform needs 0 < lo <= hi");
        tot += c.weight;
    }
    REQUIRE(tot > 0, "total component weight must be > 0");
    p->n_comp = s->n_components;
    double run = 0.0;
    for (int i = 0; i < s->n_components; ++i) {
        const heart_spectral_component &c = s->components[i];
        run += c.weight;
        p->cumw[i] = run / tot;
        p->kind[i] = c.kind;
        p->e0[i] = c.e0_keV;
        p->width[i] = c.width_keV;
        p->lo[i] = c.lo_keV;
        p->hi[i] = c.hi_keV;
        if (c.kind == HEART_SRC_LORENTZ) p->lorentz_F0[i] = 0.5 + std::atan(-c.e0_keV / (0.5 * c.width_keV)) / kPi;
    }
    REQUIRE(unit(s->axis, p->ax), "bad source axis");
    // perpendicular basis from the world axis least aligned with the cone axis
    int j = 0;
    if (std::fabs(p->ax[1]) < std::fabs(p->ax[j])) j = 1;
    if (std::fabs(p->ax[2]) < std::fabs(p->ax[j])) j = 2;
    double e[3] = {0, 0, 0};
    e[j] = 1.0;
    double t[3];
    cross(e, p->ax, t);
    unit(t, p->b1);
    cross(p->ax, p->b1, p->b2);
    for (int i = 0; i < 3; ++i) p->origin[i] = s->origin_mm[i];
    double h = std::sin(0.5 * s->cone_half_angle_rad);
    p->one_minus_cos_max = 2.0 * h * h;
    p->sig1 = s->spot_fwhm_mm[0] / (2.0 * std::sqrt(2.0 * kLn2));
    p->sig2 = s->spot_fwhm_mm[1] / (2.0 * std::sqrt(2.0 * kLn2));
    REQUIRE(finite3(s->polarization), "non-finite polarisation");
    p->pol_on = unit(s->polarization, p->pol) ? 1 : 0;
    bool table = false;
    for (int i = 0; i < s->n_components; ++i) table |= s->components[i].kind == HEART_SRC_TABLE;
    if (table) {
        REQUIRE(spectrum, "tabulated spectra need a device copy this entry point cannot make");
        const int n = s->n_table;
        REQUIRE(s->table_keV && s->table_pdf && n >= 2 && n <= kMaxTable, "spectrum table: 2..8192 knots");
        const double *x = s->table_keV, *f = s->table_pdf;
        for (int i = 0; i < n; ++i) {
            REQUIRE(std::isfinite(x[i]) && std::isfinite(f[i]) && f[i] >= 0.0, "spectrum table: finite, pdf >= 0");
            if (i > 0) REQUIRE(x[i] > x[i - 1], "spectrum table: knots must ascend");
        }
        REQUIRE(x[0] > 0.0, "spectrum table: energies must be > 0");
        // CDF at the knots by the trapezoid rule, in this order of operations
        std::vector<double> C((size_t)n);
        double run = 0.0, first = 0.0;
        C[0] = 0.0;
        for (int i = 0; i + 1 < n; ++i) {
            const double m = 0.5 * (f[i] + f[i + 1]) * (x[i + 1] - x[i]);
            run += m;
            first += m * (0.5 * (x[i] + x[i + 1]));       // the interval's mean energy
            C[i + 1] = run;
        }
        REQUIRE(run > 0.0 && std::isfinite(run), "spectrum table has no mass");
        for (int i = 1; i < n; ++i) C[i] /= run;
        C[n - 1] = 1.0;
        p->n_tab = n;
        p->tab_mean = first / run;
        spectrum->assign(spectrum_bytes(n), 0);
        unsigned char *b = spectrum->data();
        double *cdf = (double *)b, *keV = (double *)(b + 8 * (size_t)n);
        unsigned long long *thr = (unsigned long long *)(b + 16 * (size_t)n);
        float *off = (float *)(b + 24 * (size_t)n), *inv = (float *)(b + 28 * (size_t)n);
        float *dE = (float *)(b + 32 * (size_t)n), *w = (float *)(b + 36 * (size_t)n);
        for (int i = 0; i < n; ++i) {
            cdf[i] = C[i];
            keV[i] = x[i];
            // (word + 1/2) 2^-32 < C  <=>  word < ceil(C 2^32 - 1/2): the FP64 decision on words
            const double t = std::ceil(C[i] * 4294967296.0 - 0.5);
            thr[i] = t <= 0.0 ? 0ull : (unsigned long long)t;
            off[i] = (float)((double)thr[i] + 0.5 - C[i] * 4294967296.0);   // in [0, 1)
            inv[i] = (i + 1 < n && C[i + 1] > C[i]) ? (float)(1.0 / ((C[i + 1] - C[i]) * 4294967296.0)) : 0.0f;
            dE[i] = (float)(x[i] - p->tab_mean);
            w[i] = i + 1 < n ? (float)(x[i + 1] - x[i]) : 0.0f;
        }
    }
#undef REQUIRE
    return HEART_OK;
}

heart_status build_ray_params(const heart_ray_arrays *r, SourceParams *p, char *err, int errlen) {
    std::memset(p, 0, sizeof *p);
#define REQUIRE(cond, msg) do { if (!(cond)) { set_err(err, errlen, msg); return HEART_EINVAL; } } while (0)
    REQUIRE(r, "null ray arrays");
    REQUIRE(r->origin_x && r->origin_y && r->origin_z && r->dir_x && r->dir_y && r->dir_z && r->energy_keV,
            "null ray array");
    const bool any = r->pol_x || r->pol_y || r->pol_z, all = r->pol_x && r->pol_y && r->pol_z;
    REQUIRE(!any || all, "polarisation needs all three arrays or none");
    const double *a[10] = {r->origin_x, r->origin_y, r->origin_z, r->dir_x, r->dir_y, r->dir_z, r->energy_keV,
                           r->pol_x, r->pol_y, r->pol_z};
    for (int i = 0; i < 10; ++i) {
        REQUIRE(((uintptr_t)a[i] % 8) == 0, "ray arrays must be 8-byte aligned");
        p->ray[i] = a[i];
    }
    p->user = 1;
    p->pol_on = all ? 1 : 0;
    // a single nominal component so that per-component tables stay defined
    p->n_comp = 1;
    p->kind[0] = HEART_SRC_MONO;
    p->e0[0] = 8.0;
    p->cumw[0] = 1.0;
    p->ax[2] = 1.0;
    p->b1[0] = 1.0;
    p->b2[1] = 1.0;
#undef REQUIRE
    return HEART_OK;
}

heart_status build_qe_params(const heart_qe_table *q, unsigned long long *eimg, QeParams *p, char *err,
                             int errlen) {
    std::memset(p, 0, sizeof *p);
    p->eimg = eimg;
    if (!q || q->n == 0) return HEART_OK;
#define REQUIRE(cond, msg) do { if (!(cond)) { set_err(err, errlen, msg); return HEART_EINVAL; } } while (0)
    REQUIRE(q->n > 0 && q->n <= kMaxQe, "QE table needs 1..32 knots");
    REQUIRE(q->keV && q->qe, "null QE arrays");
    for (int i = 0; i < q->n; ++i) {
        REQUIRE(std::isfinite(q->keV[i]) && q->keV[i] > 0, "QE knot energies must be > 0");
        REQUIRE(q->qe[i] >= 0 && q->qe[i] <= 1, "QE values must be in [0, 1]");
        REQUIRE(i == 0 || q->keV[i] > q->keV[i - 1], "QE knot energies must increase");
        p->keV[i] = q->keV[i];
        p->qe[i] = q->qe[i];
    }
    p->n = q->n;
#undef REQUIRE
    return HEART_OK;
}

}  // namespace heart
