/*
 * oracle.c -- plain FP64 CPU oracle of the HEART mosaic-crystal ray path.
 *
 * TEST INFRASTRUCTURE ONLY (see heart_oracle.h).  Slow and literal on purpose.
 *
 * What is computed (Gawne et al., "HEART: A New X-Ray Tracing Code for Mosaic
 * Crystal Spectrometers", arXiv 2503.16955):
 *
 *  Source (Sec. 2.1; uniform emission in solid angle, Sec. 4.2):
 *    energy from a weighted mixture of spectral components, origin = source
 *    point + 2-D Gaussian spot, direction uniform in solid angle inside a cone.
 *  Per-ray constants: Bragg angle from Eq. (BraggLaw), hc/E = 2 d sin(aB);
 *    mu0 from an absorption length; Q = |r_e F_H / V|^2 lambda^3 / sin(2 aB)
 *    (Sec. 2.2.3); majorant mubar = mu0 + Q * max R.
 *  Entry (Sec. 2.2.3 first paragraph): a ray that misses the crystal's front
 *    face is discarded.
 *  Walk (Sec. 2.2.4, Eq. AnyEvent, Eq. ReflXsection, Appendix A Method II):
 *    the reflection rate of Eq. (ReflXsection) equals Q * E_{n ~ f}[R(Delta) G(a~)]
 *    when the crystallite normal n is drawn from the MDF f on the unit sphere,
 *    because the cos(aB + Delta) factor of that equation is the Jacobian
 *    dOmega_n = cos(a~) dDelta dpsi.  Free paths are therefore drawn with the
 *    constant rate mubar (null-collision / delta tracking); at each tentative
 *    collision the ray is absorbed with probability mu0/mubar, otherwise a
 *    crystallite normal n is drawn from the MDF about the local surface normal
 *    and accepted with probability R(Delta) G_unpol(a~) / max R, where
 *    a~ = asin|k.n| (both H and H-bar, Sec. 2.2.3 last part) and
 *    Delta = a~ - aB - Delta_M.  On acceptance k <- k - 2 (k.n) n (reflection
 *    equation of Sec. 2.2.4).  The walk ends at the first boundary crossing of
 *    the free path (exit), at absorption, at the (n_max+1)-th reflection
 *    (CAPPED) or at the per-ray collision cap (STUCK).
 *  No rocking curve (Sec. 2.2.1, IRC "none"): R(Delta) = delta(Delta).  Only
 *    crystallites at exactly a~0 = aB + Delta_M reflect; their normals lie on
 *    the two cones k.n = -/+ sin a~0 about k, and with dOmega = cos a~ da~ dpsi
 *    the rate becomes Q cos a~0 sum_cones int_0^2pi f(n(psi)) G dpsi.  The
 *    candidates then carry the bound Q cos a~0 * 2 cones * 2 pi f(0) instead of
 *    Q max R, and a candidate picks a cone and a uniform psi and is kept with
 *    probability f(n) G / f(0) (f from the MDF's own formula).  The thinned
 *    sampler bounds each cone per straight segment instead: the cone facing
 *    the ray by f at the tilt 2 sin^2(d/2) (d: distance of sin a~0 from the
 *    segment's |k.N| range), the other by f at 2 sin^2(a~0/2).  On the
 *    facing cone the tilt grows with the azimuth psi measured from the side
 *    of N, q(psi) = q0 + cos(a~0) cos(g) (1 - cos psi) (sin g = |k.N|), so
 *    outside a window |psi| < psi* the MDF is below v* f(0) (v* the thinning
 *    level, q_v the tilt where W / W(0) falls to v*): the facing cone splits
 *    into the window (bound f at 2 sin^2(d/2)) and the rest (bound v* f(0)).
 *    A candidate takes the window, the rest or the other cone by its share
 *    of the bound, psi uniform over that part, and is kept with
 *    f(n) G / (that part's bound).
 *  Detector (Sec. 2.3): exiting rays are propagated to the detector plane and
 *    binned into integer pixel counts.
 *
 * Random numbers: one Philox4x32-10 block per call; key = seed, counter =
 * (ray_lo, ray_hi, call, 0).  Call 0: component, component parameter, cone
 * cosine, cone azimuth.  Call 1: spot Box-Muller pair, energy Box-Muller pair.
 * Calls 2, 3, ...: one per free-path draw (u0 path, u1 absorb/accept, u2 MDF
 * quantile, u3 azimuth).  A 32-bit word w maps to u = (w + 0.5) 2^-32.
 */
#define _GNU_SOURCE
#include "heart_oracle.h"

#include <complex.h>
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define HC_KEV_A 12.398419843320026   /* h c in keV Angstrom (SI 2019 exact) */
#define PI 3.14159265358979323846
#define LN2 0.69314718055994530942

static __thread char g_err[256];
const char *orc_last_error(void) { return g_err; }
static int fail(const char *m) { snprintf(g_err, sizeof g_err, "%s", m); return -1; }

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1]*b[2] - a[2]*b[1];
    c[1] = a[2]*b[0] - a[0]*b[2];
    c[2] = a[0]*b[1] - a[1]*b[0];
}
static int normalize3(double a[3]) {
    double n = sqrt(dot3(a, a));
    if (!(n > 0)) return -1;
    a[0] /= n; a[1] /= n; a[2] /= n;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.2):        */
/* S-box round on (x0,x1,x2,x3) with key (k0,k1):                      */
/*   hi0:lo0 = M0*x0, hi1:lo1 = M1*x2,                                  */
/*   out = (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0);                    */
/* the key is bumped by the Weyl constants between rounds.             */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static double U(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* ------------------------------------------------------------------ */
/* adaptive Gauss-Legendre quadrature.  The 20 nodes are the roots of  */
/* the Legendre polynomial P_20, found once by Newton's method on the  */
/* three-term recurrence; weights 2 / ((1 - x^2) P_20'(x)^2).           */
/* ------------------------------------------------------------------ */
typedef double (*fn_t)(const void *ctx, double x);

#define GL_N 20
static double gl_x[GL_N], gl_w[GL_N];
static pthread_once_t gl_once = PTHREAD_ONCE_INIT;

static void gl_init(void) {
    for (int i = 0; i < GL_N; ++i) {
        double x = cos(PI * (i + 0.75) / (GL_N + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int n = 2; n <= GL_N; ++n) {
                double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
                p0 = p1; p1 = p2;
            }
            dp = GL_N * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

static double gl_panel(fn_t f, const void *ctx, double a, double b) {
    double m = 0.5 * (a + b), h = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < GL_N; ++i) s += gl_w[i] * f(ctx, m + h * gl_x[i]);
    return s * h;
}

static double gl_adapt(fn_t f, const void *ctx, double a, double b, double whole, double rel,
                       double afloor, int depth, long *budget) {
    double m = 0.5 * (a + b);
    double l = gl_panel(f, ctx, a, m), r = gl_panel(f, ctx, m, b);
    *budget -= 2 * GL_N;
    double both = l + r;
    double tol = rel * fabs(both);
    if (tol < afloor) tol = afloor;
    if (fabs(both - whole) <= tol || depth <= 0 || *budget <= 0 || !(m > a && b > m))
        return both;
    return gl_adapt(f, ctx, a, m, l, rel, 0.5 * afloor, depth - 1, budget) +
           gl_adapt(f, ctx, m, b, r, rel, 0.5 * afloor, depth - 1, budget);
}

/* integral of f over [a,b], each sub-interval refined until two successive
 * Gauss-Legendre estimates agree to relative tolerance rel (floor 4e-16) or
 * to the absolute tolerance afloor */
static double integrate_abs(fn_t f, const void *ctx, double a, double b, double rel, double afloor) {
    pthread_once(&gl_once, gl_init);
    if (!(b > a)) return 0.0;
    if (rel < 4e-16) rel = 4e-16;
    long budget = 4000000;
    const int n = 4;
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        double x0 = a + (b - a) * i / n, x1 = (i == n - 1) ? b : a + (b - a) * (i + 1) / n;
        total += gl_adapt(f, ctx, x0, x1, gl_panel(f, ctx, x0, x1), rel, afloor / n, 40, &budget);
    }
    return total;
}

static double integrate(fn_t f, const void *ctx, double a, double b, double rel) {
    return integrate_abs(f, ctx, a, b, rel, 1e-300);
}

/* ------------------------------------------------------------------ */
/* intrinsic rocking curve (Sec. 2.2.1), unit area in Delta            */
/* ------------------------------------------------------------------ */
void orc_pv_width(double fg, double fl, double *fwhm, double *eta) {
    /* total FWHM (fifth-order form) and Lorentzian fraction (cubic form) */
    double s = pow(fg, 5) + 2.69269 * pow(fg, 4) * fl + 2.42843 * pow(fg, 3) * fl * fl +
               4.47163 * fg * fg * pow(fl, 3) + 0.07842 * fg * pow(fl, 4) + pow(fl, 5);
    double F = pow(s, 0.2);
    double r = fl / F;
    *fwhm = F;
    *eta = 1.36603 * r - 0.47719 * r * r + 0.11116 * r * r * r;
}

static double gauss_shape(double x, double F) {     /* Eq. (Gaussian) */
    return sqrt(4.0 * LN2 / (PI * F * F)) * exp(-4.0 * LN2 * x * x / (F * F));
}
static double lorentz_shape(double x, double F) {   /* Eq. (Lorentz) */
    return F / (2.0 * PI) / (0.25 * F * F + x * x);
}

/* Darwin curve (textbook, e.g. Als-Nielsen & McMorrow ch. 6): R = 1 on the
 * plateau |y| <= 1, (|y| - sqrt(y^2-1))^2 outside.  Written as 1/(|y|+sqrt)^2. */
static double darwin_R(double y) {
    double a = fabs(y);
    if (a <= 1.0) return 1.0;
    double d = a + sqrt(a * a - 1.0);
    return 1.0 / (d * d);
}
/* Darwin-Prins with absorption: R = |eta - sqrt(eta^2-1)|^2, eta = y + i g,
 * the root of modulus <= 1; the two roots' moduli multiply to 1. */
static double darwin_prins_R(double y, double g) {
    double complex eta = y + g * I;
    double complex z = csqrt(eta * eta - 1.0);
    double a = cabs(eta - z), b = cabs(eta + z);
    double m = a > b ? a : b;
    return 1.0 / (m * m);
}
static double dp_integrand(const void *ctx, double phi) {
    double g = *(const double *)ctx;
    double y = tan(phi);
    if (!(y < 1e150)) return 0.25;
    return darwin_prins_R(y, g) * (1.0 + y * y);
}
double orc_darwin_prins_area(double g) {
    /* 2 * integral_0^inf R(y) dy with y = tan(phi) */
    double a = integrate(dp_integrand, &g, 0.0, PI / 4, 1e-13);
    double b = integrate(dp_integrand, &g, PI / 4, PI / 2, 1e-13);
    return 2.0 * (a + b);
}

/* IRC parameters evaluated once per spectrometer */
typedef struct {
    int kind;
    double fwhm;        /* G, L, box FWHM; pV total FWHM */
    double eta;         /* pV Lorentzian fraction */
    double delta;       /* Darwin half-width: FWHM = (3/sqrt 2) delta */
    double norm;        /* Darwin / DP: delta * integral R(y) dy */
    double g;           /* DP absorption parameter */
} irc_params;

static void irc_prepare(const orc_spec *s, irc_params *p) {
    memset(p, 0, sizeof *p);
    p->kind = s->irc;
    p->fwhm = s->irc_fwhm_rad;
    p->delta = s->irc_fwhm_rad * sqrt(2.0) / 3.0;
    p->g = s->prins_g;
    if (s->irc == ORC_IRC_DARWIN) p->norm = p->delta * 8.0 / 3.0;
    if (s->irc == ORC_IRC_DARWIN_PRINS) p->norm = p->delta * orc_darwin_prins_area(s->prins_g);
    if (s->irc == ORC_IRC_PSEUDO_VOIGT) orc_pv_width(s->irc_fwhm_rad, s->irc_lorentz_fwhm_rad, &p->fwhm, &p->eta);
}

static double irc_eval(const irc_params *p, double x) {
    switch (p->kind) {
    case ORC_IRC_DARWIN: return darwin_R(x / p->delta) / p->norm;
    case ORC_IRC_DARWIN_PRINS: return darwin_prins_R(x / p->delta, p->g) / p->norm;
    case ORC_IRC_PSEUDO_VOIGT: return p->eta * lorentz_shape(x, p->fwhm) + (1.0 - p->eta) * gauss_shape(x, p->fwhm);
    case ORC_IRC_GAUSSIAN: return gauss_shape(x, p->fwhm);
    case ORC_IRC_LORENTZIAN: return lorentz_shape(x, p->fwhm);
    case ORC_IRC_BOX: return fabs(x) <= 0.5 * p->fwhm ? 1.0 / p->fwhm : 0.0;
    case ORC_IRC_NONE: return 0.0;           /* a delta function: no finite value */
    }
    return 0.0;
}

double orc_irc(const orc_spec *s, double x) {
    irc_params p;
    irc_prepare(s, &p);
    return irc_eval(&p, x);
}

double orc_irc_max(const orc_spec *s) {
    /* every curve here is symmetric and peaks at its centre */
    return orc_irc(s, 0.0);
}

/* ------------------------------------------------------------------ */
/* mosaic distribution (Sec. 2.2.2), as a function of q = 1 - cos(th)  */
/* On the sphere, q is distributed with density proportional to W.     */
/* ------------------------------------------------------------------ */
static double theta_of_q(double q) {
    if (q <= 0) return 0.0;
    if (q >= 2) return PI;
    return 2.0 * asin(sqrt(0.5 * q));
}

double orc_mdf_qmax(const orc_spec *s) {
    if (s->mdf == ORC_MDF_UNIFORM) {
        double h = sin(0.25 * s->mdf_fwhm_rad);
        return 2.0 * h * h;           /* 1 - cos(Gamma/2) */
    }
    return 2.0;
}

double orc_mdf_W(const orc_spec *s, double q) {
    double G = s->mdf_fwhm_rad;
    switch (s->mdf) {
    case ORC_MDF_GAUSSIAN: {
        double th = theta_of_q(q);
        return exp(-4.0 * LN2 * th * th / (G * G));
    }
    case ORC_MDF_LORENTZIAN: {
        double th = theta_of_q(q);
        return 1.0 / (0.25 * G * G + th * th);
    }
    case ORC_MDF_PSEUDO_VOIGT: {
        double th = theta_of_q(q);
        return s->mdf_eta * lorentz_shape(th, G) + (1.0 - s->mdf_eta) * gauss_shape(th, G);
    }
    case ORC_MDF_VMF: {            /* Eq. (MF): exp((cos th - 1)/s^2), Gamma = 2 s sqrt(2 ln 2) */
        double sg = G / (2.0 * sqrt(2.0 * LN2));
        return exp(-q / (sg * sg));
    }
    case ORC_MDF_WL:               /* Eq. (WL): 1 / ((Gamma/2)^2 + 2 - 2 cos th) */
        return 1.0 / (0.25 * G * G + 2.0 * q);
    case ORC_MDF_SWL: {            /* Eq. (SWL): 1 / (cosh(Gamma/2) - cos th)^2 */
        double sh = sinh(0.25 * G);
        double b = 2.0 * sh * sh + q;  /* cosh(G/2) - 1 + q */
        return 1.0 / (b * b);
    }
    case ORC_MDF_UNIFORM:
        return q <= orc_mdf_qmax(s) ? 1.0 : 0.0;
    }
    return 0.0;
}

static double mdf_W_cb(const void *ctx, double q) { return orc_mdf_W((const orc_spec *)ctx, q); }

/* absolute accuracy floor for MDF integrals: 1e-19 of W(0) Gamma^2 / 8, far
 * below the smallest tail mass the table resolves (2^-33 of the total) */
static double mdf_afloor(const orc_spec *s) {
    double G = s->mdf_fwhm_rad;
    return 1e-19 * orc_mdf_W(s, 0.0) * G * G / 8.0;
}
/* W(theta(q)) sin(theta) as a function of theta, for the shapes defined in
 * theta; integrating these in theta avoids the square-root end point of
 * theta(q) at q = 2 (dq = sin(theta) dtheta) */
static double mdf_Wtheta_cb(const void *ctx, double th) {
    const orc_spec *s = (const orc_spec *)ctx;
    double h = sin(0.5 * th);
    return orc_mdf_W(s, 2.0 * h * h) * sin(th);
}
static int mdf_in_theta(const orc_spec *s) {
    return s->mdf == ORC_MDF_GAUSSIAN || s->mdf == ORC_MDF_LORENTZIAN || s->mdf == ORC_MDF_PSEUDO_VOIGT;
}
static double mdf_int(const orc_spec *s, double a, double b) {
    if (mdf_in_theta(s))
        return integrate_abs(mdf_Wtheta_cb, s, theta_of_q(a), theta_of_q(b), 1e-14, mdf_afloor(s));
    return integrate_abs(mdf_W_cb, s, a, b, 1e-14, mdf_afloor(s));
}

#define MAXP 400
typedef struct {
    int n;
    double q[MAXP + 1];
    double P[MAXP];        /* panel integrals               */
    double C[MAXP + 1];    /* cumulative from q = 0          */
    double S[MAXP + 1];    /* cumulative from q = qmax down  */
} mdf_panels;

/* geometric panels in q: [0,h], [h, h r], ... up to qmax, r = 2^(1/4) */
static void mdf_make_panels(const orc_spec *s, mdf_panels *P) {
    double qmax = orc_mdf_qmax(s);
    double G = s->mdf_fwhm_rad;
    double scale = G * G / 8.0;                  /* q at theta = Gamma/2 */
    double h = 1e-6 * scale;
    if (h > qmax * 1e-6) h = qmax * 1e-6;
    int n = 0;
    P->q[0] = 0.0;
    double q = h;
    while (q < qmax && n < MAXP - 1) {
        P->q[++n] = q;
        q *= 1.189207115002721;  /* 2^(1/4) */
    }
    P->q[++n] = qmax;
    P->n = n;
    for (int i = 0; i < n; ++i) P->P[i] = mdf_int(s, P->q[i], P->q[i + 1]);
    P->C[0] = 0.0;
    for (int i = 0; i < n; ++i) P->C[i + 1] = P->C[i] + P->P[i];
    P->S[n] = 0.0;
    for (int i = n - 1; i >= 0; --i) P->S[i] = P->S[i + 1] + P->P[i];
}

double orc_mdf_norm(const orc_spec *s) {
    mdf_panels P;
    mdf_make_panels(s, &P);
    return P.C[P.n];
}

static double panels_cdf(const orc_spec *s, const mdf_panels *P, double q) {
    if (q <= 0) return 0.0;
    int k = 0;
    while (k < P->n - 1 && P->q[k + 1] <= q) ++k;
    if (q >= P->q[P->n]) return 1.0;
    return (P->C[k] + mdf_int(s, P->q[k], q)) / P->C[P->n];
}
static double panels_ccdf(const orc_spec *s, const mdf_panels *P, double q) {
    if (q <= 0) return 1.0;
    if (q >= P->q[P->n]) return 0.0;
    int k = 0;
    while (k < P->n - 1 && P->q[k + 1] <= q) ++k;
    return (P->S[k + 1] + mdf_int(s, q, P->q[k + 1])) / P->S[0];
}

double orc_mdf_cdf(const orc_spec *s, double q) {
    mdf_panels P;
    mdf_make_panels(s, &P);
    return panels_cdf(s, &P, q);
}
double orc_mdf_ccdf(const orc_spec *s, double q) {
    mdf_panels P;
    mdf_make_panels(s, &P);
    return panels_ccdf(s, &P, q);
}

/* Solve for q in panel k: either  integral_{q_k}^{q} W = r  (from_top = 0)
 * or  integral_{q}^{q_{k+1}} W = r  (from_top = 1), by safeguarded Newton. */
static double panel_solve(const orc_spec *s, const mdf_panels *P, int k, double r, int from_top) {
    double lo = P->q[k], hi = P->q[k + 1];
    if (r <= 0) return from_top ? hi : lo;
    if (r >= P->P[k]) return from_top ? lo : hi;
    double x = lo + (hi - lo) * (from_top ? 1.0 - r / P->P[k] : r / P->P[k]);
    for (int it = 0; it < 200; ++it) {
        double g = from_top ? mdf_int(s, x, P->q[k + 1]) - r
                            : mdf_int(s, P->q[k], x) - r;
        /* g is increasing in x for from_top = 0, decreasing for from_top = 1 */
        if (fabs(g) <= 1e-15 * r) break;            /* at quadrature accuracy */
        int below = from_top ? (g > 0) : (g < 0);
        if (below) lo = x; else hi = x;
        double w = orc_mdf_W(s, x);
        double step = (w > 0) ? (from_top ? g / w : -g / w) : 0.0;
        double xn = x + step;
        if (!(w > 0) || !(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - x) <= 1e-16 * fabs(x) + 1e-300 || hi - lo <= 1e-16 * hi) { x = xn; break; }
        x = xn;
    }
    return x;
}

static double panels_quantile(const orc_spec *s, const mdf_panels *P, double u) {
    double Z = P->C[P->n];
    double target = u * Z;
    int k = 0;
    while (k < P->n - 1 && P->C[k + 1] <= target) ++k;
    return panel_solve(s, P, k, target - P->C[k], 0);
}
static double panels_quantile_tail(const orc_spec *s, const mdf_panels *P, double comp) {
    /* q with 1 - F(q) = comp, computed from the top */
    double Z = P->S[0];
    double target = comp * Z;
    int k = P->n - 1;
    while (k > 0 && P->S[k] <= target) --k;
    return panel_solve(s, P, k, target - P->S[k + 1], 1);
}

double orc_mdf_quantile_exact(const orc_spec *s, double u, int tail_complement, double comp) {
    mdf_panels P;
    mdf_make_panels(s, &P);
    if (tail_complement) return panels_quantile_tail(s, &P, comp);
    return panels_quantile(s, &P, u);
}

int orc_mdf_build_table(const orc_spec *s, orc_mdf_table *t) {
    mdf_panels *P = (mdf_panels *)malloc(sizeof(mdf_panels));
    if (!P) return fail("out of memory");
    mdf_make_panels(s, P);
    if (!(P->C[P->n] > 0)) { free(P); return fail("MDF has zero mass"); }
    for (int i = 0; i < ORC_MDF_M; ++i)
        t->body[i] = (i == 0) ? 0.0 : panels_quantile(s, P, (double)i / ORC_MDF_M);
    for (int j = 0; j <= ORC_MDF_T; ++j) {
        double tau = 12.0 + 21.0 * (double)j / ORC_MDF_T;
        t->tail[j] = panels_quantile_tail(s, P, exp2(-tau));
    }
    t->tail[0] = t->body[ORC_MDF_M - 1] = panels_quantile_tail(s, P, 1.0 / ORC_MDF_M);
    t->qmax = orc_mdf_qmax(s);
    free(P);
    return 0;
}

/* Table lookup: the top 12 bits of w select a body interval (u = i / 4096),
 * the low 20 bits plus one half give the fraction inside it.  The last body
 * interval is replaced by the tail segment, linear in tau = -log2(1 - u). */
double orc_mdf_table_lookup(const orc_mdf_table *t, uint32_t w) {
    uint32_t i = w >> 20;
    if (i < ORC_MDF_M - 1) {
        double f = ((double)(w & 0xFFFFFu) + 0.5) * (1.0 / 1048576.0);
        return t->body[i] + f * (t->body[i + 1] - t->body[i]);
    }
    double m = (double)(0xFFFFFFFFu - w) + 0.5;     /* (1 - u) 2^32 */
    double tau = 32.0 - log2(m);
    double y = (tau - 12.0) * (ORC_MDF_T / 21.0);
    int j = (int)floor(y);
    if (j > ORC_MDF_T - 1) j = ORC_MDF_T - 1;
    if (j < 0) j = 0;
    double f = y - j;
    return t->tail[j] + f * (t->tail[j + 1] - t->tail[j]);
}

/* ------------------------------------------------------------------ */
/* per-ray constants                                                   */
/* ------------------------------------------------------------------ */
static double refl_K(const orc_spec *s) {
    if (s->refl_K_per_mm2 >= 0) return s->refl_K_per_mm2;
    /* Darwin half-width delta = r_e lambda^2 |F| / (pi V sin 2aB) (kinematic
     * textbook relation) => K = pi delta sin(2 aB) / lambda^2 at E_ref */
    double lam_A = HC_KEV_A / s->refl_ref_keV;
    double sb = lam_A / (2.0 * s->d_spacing_A);
    double cb = sqrt(1.0 - sb * sb);
    double lam_mm = lam_A * 1e-7;
    double delta = s->refl_darwin_fwhm_rad * sqrt(2.0) / 3.0;
    return PI * delta * (2.0 * sb * cb) / (lam_mm * lam_mm);
}

/* the energy-dependent rocking curve at E: width scale and added peak shift,
 * linear between the knots and constant beyond them */
static void irc_energy(const orc_spec *s, double E, double *wscale, double *shift) {
    *wscale = 1.0;
    *shift = 0.0;
    int n = s->n_irc_e;
    if (n <= 0) return;
    const double *x = s->irc_e_keV;
    if (n == 1 || E <= x[0]) { *wscale = s->irc_e_wscale[0]; *shift = s->irc_e_shift_rad[0]; return; }
    if (E >= x[n - 1]) { *wscale = s->irc_e_wscale[n - 1]; *shift = s->irc_e_shift_rad[n - 1]; return; }
    int i = 0;
    while (!(E < x[i + 1])) ++i;
    double f = (E - x[i]) / (x[i + 1] - x[i]);
    *wscale = s->irc_e_wscale[i] + f * (s->irc_e_wscale[i + 1] - s->irc_e_wscale[i]);
    *shift = s->irc_e_shift_rad[i] + f * (s->irc_e_shift_rad[i + 1] - s->irc_e_shift_rad[i]);
}

/* the reflection orders of a spectrometer: multiple m, K ratio, width ratio */
static int spec_orders(const orc_spec *s, int m[ORC_MAX_ORDERS], double kr[ORC_MAX_ORDERS],
                       double wr[ORC_MAX_ORDERS]) {
    if (s->n_orders <= 0) { m[0] = 1; kr[0] = 1.0; wr[0] = 1.0; return 1; }
    int n = s->n_orders > ORC_MAX_ORDERS ? ORC_MAX_ORDERS : s->n_orders;
    for (int h = 0; h < n; ++h) { m[h] = s->order_m[h]; kr[h] = s->order_K_rel[h]; wr[h] = s->order_w_rel[h]; }
    return n;
}

/* no rocking curve: the scatter-candidate rate of an order is Q cos a~0 times
 * 2 cones x 2 pi f(0), f = W / (2 pi int W dq) the MDF per unit solid angle;
 * this returns 2 * 2 pi f(0) = 2 W(0) / int W dq */
static double none_factor(const orc_spec *s) {
    return 2.0 * orc_mdf_W(s, 0.0) / orc_mdf_norm(s);
}

static int ray_constants(const orc_spec *s, double E, double none_fac, orc_ray_consts *c);

int orc_ray_constants(const orc_spec *s, double E, orc_ray_consts *c) {
    return ray_constants(s, E, s->irc == ORC_IRC_NONE ? none_factor(s) : 0.0, c);
}

static int ray_constants(const orc_spec *s, double E, double none_fac, orc_ray_consts *c) {
    memset(c, 0, sizeof *c);
    c->E_keV = E;
    c->lambda_A = HC_KEV_A / E;
    c->mu0 = 1.0 / (s->absorption_length_mm * pow(E / s->absorption_ref_keV, s->absorption_power));
    int m[ORC_MAX_ORDERS];
    double kr[ORC_MAX_ORDERS], wr[ORC_MAX_ORDERS], wscale, shift;
    c->n_orders = spec_orders(s, m, kr, wr);
    irc_energy(s, E, &wscale, &shift);
    c->shift_rad = s->irc_shift_rad + shift;
    double K = refl_K(s), rmax = orc_irc_max(s), lam_mm = c->lambda_A * 1e-7;
    double qr_sum = 0.0;
    c->no_bragg = 1;
    for (int h = 0; h < c->n_orders; ++h) {
        /* Eq. (BraggLaw) on the planes d / m_h */
        double sb = m[h] * c->lambda_A / (2.0 * s->d_spacing_A);
        c->ord_sin[h] = sb;
        c->ord_w[h] = wr[h] * wscale;
        if (!(sb < 1.0)) {
            c->ord_alpha[h] = NAN;
            continue;
        }
        c->no_bragg = 0;
        c->ord_alpha[h] = asin(sb);
        double cb = sqrt(1.0 - sb * sb);
        double Kh = K * kr[h];
        c->ord_Q[h] = Kh * Kh * lam_mm * lam_mm * lam_mm / (2.0 * sb * cb);
        c->ord_qr[h] = c->ord_Q[h] * (rmax / c->ord_w[h]);   /* a curve w times as wide peaks 1/w as high */
        if (s->irc == ORC_IRC_NONE) {
            double a0 = c->ord_alpha[h] + c->shift_rad;          /* the only reflecting incidence */
            c->ord_qr[h] = (a0 > 0.0 && a0 < 0.5 * PI) ? c->ord_Q[h] * cos(a0) * none_fac : 0.0;
        }
        qr_sum += c->ord_qr[h];
    }
    c->sin_aB = c->ord_sin[0];
    c->alpha_B = c->ord_alpha[0];
    c->Q = c->ord_Q[0];
    c->mubar = c->mu0 + qr_sum;
    c->p_abs = c->mu0 / c->mubar;
    return 0;
}

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_spec *s;
    /* flat frame */
    double N[3], ed[3], en[3];
    /* cylinder frame */
    double ax[3], cc[3], ww[3], sphi, cphi;
    /* detector frame */
    double eu[3], ev[3], nd[3];
    double irc_max;
    irc_params irc;
    orc_mdf_table *mdf;
    /* thinned sampler: v* and the IRC half-width X* beyond which R/R_max <= v* */
    double vstar, xstar;
    /* no rocking curve: the factor of none_factor() and W(0); thinned: the tilt
     * q_v beyond which W / W(0) <= v* (INFINITY if W never falls that low) */
    int irc_none;
    double none_fac, W0, none_qv;
} geom;

/* q_v: a tilt with W(q) / W(0) <= v* for every q >= q_v (the MDFs decrease
 * with the tilt), by 100 bisection steps on [0, 2] and widened by 1e-9
 * relative; INFINITY if W(2) / W(0) > v*. */
static double none_tilt(const orc_spec *s, double W0, double vstar) {
    if (orc_mdf_W(s, 2.0) / W0 > vstar) return INFINITY;
    double lo = 0.0, hi = 2.0;
    for (int i = 0; i < 100; ++i) {
        double m = 0.5 * (lo + hi);
        if (orc_mdf_W(s, m) / W0 <= vstar) hi = m; else lo = m;
    }
    return hi * (1.0 + 1e-9);
}

/* X*: the smallest |x| such that R(x') / R_max <= v* for every |x'| >= X*.
 * Found by scanning |x| down from 1 rad on a geometric grid (ratio 1.0005),
 * then bisecting the last crossing; widened by 1e-6 relative. */
static double irc_xstar(const irc_params *p, double rmax, double vstar) {
    double hi = 1.0;
    if (irc_eval(p, hi) / rmax > vstar || irc_eval(p, -hi) / rmax > vstar) return -1.0;
    double x = hi;
    for (;;) {
        double y = x / 1.0005;
        if (y < 1e-12) return 1e-12;
        if (irc_eval(p, y) / rmax > vstar || irc_eval(p, -y) / rmax > vstar) {
            double lo = y, up = x;                /* above vstar at lo, below at up */
            for (int it = 0; it < 200 && up - lo > 1e-15 * up; ++it) {
                double m = 0.5 * (lo + up);
                if (irc_eval(p, m) / rmax > vstar || irc_eval(p, -m) / rmax > vstar) lo = m; else up = m;
            }
            return up * (1.0 + 1e-6);
        }
        x = y;
    }
}

static int geom_init(geom *g, const orc_spec *s) {
    memset(g, 0, sizeof *g);
    g->s = s;
    if (s->geometry == ORC_FLAT) {
        memcpy(g->N, s->normal, sizeof g->N);
        if (normalize3(g->N)) return fail("bad normal");
        double d = dot3(s->axis, g->N);
        for (int i = 0; i < 3; ++i) g->ed[i] = s->axis[i] - d * g->N[i];
        if (normalize3(g->ed)) return fail("bad dispersive axis");
        cross3(g->N, g->ed, g->en);
    } else if (s->geometry == ORC_CYL) {
        memcpy(g->ax, s->axis, sizeof g->ax);
        if (normalize3(g->ax)) return fail("bad axis");
        double d = dot3(s->normal, g->ax);
        for (int i = 0; i < 3; ++i) g->cc[i] = s->normal[i] - d * g->ax[i];
        if (normalize3(g->cc)) return fail("bad centre direction");
        cross3(g->ax, g->cc, g->ww);
        double half = 0.5 * s->size_nondisp_mm / s->radius_mm;
        if (!(half > 0 && half < 0.5 * PI)) return fail("arc must be shorter than pi R");
        g->sphi = sin(half);
        g->cphi = cos(half);
    } else {
        return fail("bad geometry");
    }
    memcpy(g->eu, s->det_u, sizeof g->eu);
    if (normalize3(g->eu)) return fail("bad detector u");
    double d = dot3(s->det_v, g->eu);
    for (int i = 0; i < 3; ++i) g->ev[i] = s->det_v[i] - d * g->eu[i];
    if (normalize3(g->ev)) return fail("bad detector v");
    cross3(g->eu, g->ev, g->nd);
    irc_prepare(s, &g->irc);
    g->irc_max = irc_eval(&g->irc, 0.0);
    if (s->n_orders < 0 || s->n_orders > ORC_MAX_ORDERS) return fail("0..4 reflection orders");
    for (int h = 0; h < s->n_orders; ++h)
        if (s->order_m[h] < 1 || !(s->order_K_rel[h] >= 0) || !(s->order_w_rel[h] > 0) ||
            !isfinite(s->order_K_rel[h]) || !isfinite(s->order_w_rel[h]))
            return fail("order: multiple >= 1, K ratio >= 0, width ratio > 0");
    if (s->n_irc_e < 0 || s->n_irc_e > ORC_MAX_IRC_E) return fail("0..16 energy knots of the rocking curve");
    for (int i = 0; i < s->n_irc_e; ++i) {
        if (!(s->irc_e_wscale[i] > 0) || !isfinite(s->irc_e_wscale[i]) || !isfinite(s->irc_e_shift_rad[i]))
            return fail("rocking-curve energy knots: width scale > 0, finite shift");
        if (i > 0 && !(s->irc_e_keV[i] > s->irc_e_keV[i - 1])) return fail("rocking-curve energy knots must ascend");
    }
    if (s->irc == ORC_IRC_NONE) {
        /* candidates on the Bragg cones; the thinned bounds (which need X*) do not apply */
        g->irc_none = 1;
        g->W0 = orc_mdf_W(s, 0.0);
        g->none_fac = none_factor(s);
        if (!(g->W0 > 0) || !(g->none_fac > 0) || !isfinite(g->none_fac)) return fail("MDF has no mass at theta = 0");
        if (s->sampler != ORC_SAMPLER_PLAIN && s->sampler != ORC_SAMPLER_THINNED) return fail("unknown sampler");
        if (s->sampler == ORC_SAMPLER_THINNED) {
            g->vstar = s->thin_vstar > 0 ? s->thin_vstar : 1.0 / 64.0;
            if (!(g->vstar < 1.0)) return fail("thin_vstar must be < 1");
            g->none_qv = none_tilt(s, g->W0, g->vstar);
        }
    } else if (s->sampler == ORC_SAMPLER_THINNED) {
        g->vstar = s->thin_vstar > 0 ? s->thin_vstar : 1.0 / 64.0;
        if (!(g->vstar < 1.0)) return fail("thin_vstar must be < 1");
        g->xstar = irc_xstar(&g->irc, g->irc_max, g->vstar);
        if (!(g->xstar > 0)) return fail("rocking curve never drops below v*");
    } else if (s->sampler != ORC_SAMPLER_PLAIN) {
        return fail("unknown sampler");
    }
    return 0;
}

/* entry point on the front face; returns 1 on a hit */
static int entry(const geom *g, const double o[3], const double k[3], double p[3]) {
    const orc_spec *s = g->s;
    double rel[3] = {o[0] - s->centre[0], o[1] - s->centre[1], o[2] - s->centre[2]};
    if (s->geometry == ORC_FLAT) {
        double h0 = dot3(rel, g->N), kN = dot3(k, g->N);
        if (!(kN < 0) || !(h0 > 0)) return 0;
        double t = h0 / (-kN);
        for (int i = 0; i < 3; ++i) p[i] = o[i] + t * k[i];
        double r2[3] = {p[0] - s->centre[0], p[1] - s->centre[1], p[2] - s->centre[2]};
        double a = dot3(r2, g->ed), b = dot3(r2, g->en);
        if (fabs(a) > 0.5 * s->size_disp_mm || fabs(b) > 0.5 * s->size_nondisp_mm) return 0;
        return 1;
    }
    double X = dot3(rel, g->cc), Y = dot3(rel, g->ww);
    double kX = dot3(k, g->cc), kY = dot3(k, g->ww);
    double R = s->radius_mm;
    double c = X * X + Y * Y - R * R;
    if (!(c < 0)) return 0;                          /* origin must be inside r < R */
    double a = kX * kX + kY * kY;
    if (!(a > 0)) return 0;
    double b = X * kX + Y * kY;
    double sq = sqrt(b * b - a * c);
    double t = (b > 0) ? -c / (b + sq) : (-b + sq) / a;  /* the positive root */
    for (int i = 0; i < 3; ++i) p[i] = o[i] + t * k[i];
    double r2[3] = {p[0] - s->centre[0], p[1] - s->centre[1], p[2] - s->centre[2]};
    double z = dot3(r2, g->ax);
    double Xp = dot3(r2, g->cc), Yp = dot3(r2, g->ww);
    if (fabs(z - s->centre_axial_mm) > 0.5 * s->size_disp_mm) return 0;
    if (fabs(Yp) * g->cphi > Xp * g->sphi) return 0;
    return 1;
}

/* distance along k from p (inside) to the first boundary crossing */
static double exit_distance(const geom *g, const double p[3], const double k[3], int *face) {
    const orc_spec *s = g->s;
    double rel[3] = {p[0] - s->centre[0], p[1] - s->centre[1], p[2] - s->centre[2]};
    double best = INFINITY;
    int f = ORC_EXIT_SIDE;
#define CAND(val, fc) do { double v_ = (val); if (v_ < 0) v_ = 0; if (v_ < best) { best = v_; f = (fc); } } while (0)
    if (s->geometry == ORC_FLAT) {
        double h = dot3(rel, g->N), a = dot3(rel, g->ed), b = dot3(rel, g->en);
        double kh = dot3(k, g->N), ka = dot3(k, g->ed), kb = dot3(k, g->en);
        if (kh > 0) CAND((0.0 - h) / kh, ORC_EXIT_FRONT);
        if (kh < 0) CAND((-s->thickness_mm - h) / kh, ORC_EXIT_BACK);
        double Wa = 0.5 * s->size_disp_mm, Wb = 0.5 * s->size_nondisp_mm;
        if (ka > 0) CAND((Wa - a) / ka, ORC_EXIT_SIDE);
        if (ka < 0) CAND((-Wa - a) / ka, ORC_EXIT_SIDE);
        if (kb > 0) CAND((Wb - b) / kb, ORC_EXIT_SIDE);
        if (kb < 0) CAND((-Wb - b) / kb, ORC_EXIT_SIDE);
    } else {
        double z = dot3(rel, g->ax), X = dot3(rel, g->cc), Y = dot3(rel, g->ww);
        double kz = dot3(k, g->ax), kX = dot3(k, g->cc), kY = dot3(k, g->ww);
        double R = s->radius_mm, Ro = s->radius_mm + s->thickness_mm;
        double a = kX * kX + kY * kY, b = X * kX + Y * kY;
        if (a > 0) {
            double ci = X * X + Y * Y - R * R;       /* inner face r = R */
            if (b < 0) {
                double disc = b * b - a * ci;
                if (disc >= 0) CAND(ci / (-b + sqrt(disc)), ORC_EXIT_FRONT);
            }
            double co = X * X + Y * Y - Ro * Ro;     /* outer face r = R + t */
            double disc = b * b - a * co;
            if (disc < 0) disc = 0;
            double sq = sqrt(disc);
            CAND((b > 0) ? -co / (b + sq) : (-b + sq) / a, ORC_EXIT_BACK);
        }
        double zc = s->centre_axial_mm, L = 0.5 * s->size_disp_mm;
        if (kz > 0) CAND((zc + L - z) / kz, ORC_EXIT_SIDE);
        if (kz < 0) CAND((zc - L - z) / kz, ORC_EXIT_SIDE);
        double gp = -X * g->sphi + Y * g->cphi, rp = -kX * g->sphi + kY * g->cphi;
        if (rp > 0) CAND(-gp / rp, ORC_EXIT_SIDE);
        double gm = -X * g->sphi - Y * g->cphi, rm = -kX * g->sphi - kY * g->cphi;
        if (rm > 0) CAND(-gm / rm, ORC_EXIT_SIDE);
    }
#undef CAND
    *face = f;
    return best;
}

/* local surface normal N(x) (out of the front face) and tangent basis */
static void local_frame(const geom *g, const double p[3], double N[3], double t1[3], double t2[3]) {
    const orc_spec *s = g->s;
    if (s->geometry == ORC_FLAT) {
        memcpy(N, g->N, 3 * sizeof(double));
        memcpy(t1, g->ed, 3 * sizeof(double));
        memcpy(t2, g->en, 3 * sizeof(double));
        return;
    }
    double rel[3] = {p[0] - s->centre[0], p[1] - s->centre[1], p[2] - s->centre[2]};
    double X = dot3(rel, g->cc), Y = dot3(rel, g->ww);
    double r = sqrt(X * X + Y * Y);
    for (int i = 0; i < 3; ++i) N[i] = -(X * g->cc[i] + Y * g->ww[i]) / r;  /* toward the axis */
    memcpy(t1, g->ax, 3 * sizeof(double));
    cross3(N, t1, t2);
}

static void detector(const geom *g, const double x[3], const double k[3], orc_record *rec) {
    const orc_spec *s = g->s;
    rec->u_mm = NAN; rec->v_mm = NAN; rec->ix = -1; rec->iy = -1; rec->det_hit = 0;
    double den = dot3(k, g->nd);
    if (den == 0) return;
    double rel[3] = {s->det_centre[0] - x[0], s->det_centre[1] - x[1], s->det_centre[2] - x[2]};
    double t = dot3(rel, g->nd) / den;
    if (!(t > 0)) return;
    double P[3] = {x[0] + t * k[0] - s->det_centre[0], x[1] + t * k[1] - s->det_centre[1],
                   x[2] + t * k[2] - s->det_centre[2]};
    double u = dot3(P, g->eu), v = dot3(P, g->ev);
    rec->u_mm = u; rec->v_mm = v;
    double fx = u / s->pixel_mm + 0.5 * s->det_nx;
    double fy = v / s->pixel_mm + 0.5 * s->det_ny;
    if (fx >= 0 && fx < s->det_nx && fy >= 0 && fy < s->det_ny) {
        rec->ix = (int32_t)floor(fx);
        rec->iy = (int32_t)floor(fy);
        rec->det_hit = 1;
    }
}

/* ------------------------------------------------------------------ */
/* random-word source: Philox per ray, or injected words               */
/* ------------------------------------------------------------------ */
typedef struct {
    const uint32_t *words; int64_t n, pos;   /* injected if words != NULL */
    uint32_t key[2]; uint64_t ray; uint32_t call;
} wsrc;

static int next4(wsrc *ws, uint32_t w[4]) {
    if (ws->words) {
        if (ws->pos + 4 > ws->n) return 0;
        memcpy(w, ws->words + ws->pos, 4 * sizeof(uint32_t));
        ws->pos += 4;
        return 1;
    }
    uint32_t ctr[4] = {(uint32_t)ws->ray, (uint32_t)(ws->ray >> 32), ws->call++, 0u};
    orc_philox4x32_10(ctr, ws->key, w);
    return 1;
}

/* ------------------------------------------------------------------ */
/* thinned candidates: bounds of one straight segment                  */
/* ------------------------------------------------------------------ */
/* The scatter candidates (rate Q R_max, marks: the acceptance uniform v and
 * the crystallite normal n) split by their marks into independent Poisson
 * processes (marking theorem):
 *   (a) v < v*: every candidate, tested as usual;
 *   (b) v >= v*, q(n) in [q_min, 2 - q_min] and the azimuth of n in the arcs
 *       where |Delta| < X*: tested as usual;
 *   (c) the rest, which cannot reflect: with |Delta| >= X*, R / R_max <= v* <= v.
 * On a straight segment the ray's grazing angle stays in [a_lo, a_hi]; a
 * crystallite tilted by theta has asin|k.n| within theta of it, so if
 * theta < d - X* (d <= the distance of alpha_B + Delta_M from [a_lo, a_hi])
 * then |Delta| >= X*.  d is taken between the sines, which is never larger
 * than between the angles (asin has slope >= 1).  Process (c) is never
 * generated.  Process (b) is generated at rate Q R_max (1 - v*) P_A pbar:
 * n's table word uniform over [w0, 2^32) (mass P_A), w0 the first word of
 * the table interval holding the grid point q_j = 2^(j/8 - 48) just below
 * q_min; then kept with probability P_xi(theta) / pbar (P_xi: the arc
 * measure, pbar >= P_xi on the segment), its azimuth uniform over the arcs.
 * A segment with d <= X* keeps the plain candidate stream (v* = 1).
 * pbar is the arc measure's bound at the smallest tilt, where the window can
 * sit at the edge of cos(xi') and the measure is largest; with one reflection
 * order, process (b) is split further by the tilt (marking theorem again):
 * band B, the table words [w1, w2) of the tilts from the grid point 12 steps
 * above q_min's (a factor 2^1.5 in q) to q_J = 2^(-33/8) (0.34 rad), where the
 * window stays away from the edge, is generated at its own bound pbarB < pbar;
 * band A, the words [w0, w1) and [w2, 2^32), at pbar.  A (b) candidate falls in
 * band A with probability sA = P_A pbar / (P_A pbar + P_B pbarB). */
typedef struct {
    double ra, vstar;         /* share of process (a) among the order's scatter candidates, its v range */
    double qmin, pbar;        /* process (b): tilt bound and arc-measure bound */
    double S1, S2;            /* |k.n| window of |Delta| < X* */
    uint64_t w0, wspan;       /* process (b): table words [w0, w0 + wspan) */
    uint64_t w1, w2;          /* band B: table words [w1, w2) (w1 = w2 = w0: no band B) */
    double pbarB, sA;         /* band B's arc-measure bound; band A's share of process (b) */
    double lam;               /* the order's candidate rate on the segment */
    /* no rocking curve, thinned: W at the smallest tilt each Bragg cone can
     * reach on the segment, relative to W(0); the facing cone's window |psi| <
     * psis; the cumulative shares of the window and of the whole facing cone */
    double wn, wf, psis, pin, pio;
} order_bound;

typedef struct {
    double mu, pa;            /* majorant of the segment and the absorption share mu0 / mu */
    int n;                    /* reflection orders */
    double cum[ORC_MAX_ORDERS];   /* cumulative shares of the orders among scatter candidates */
    order_bound o[ORC_MAX_ORDERS];
} seg_bound;

/* first word of the table interval containing q (conservative lower end) */
static uint64_t word_floor(const orc_mdf_table *t, double q) {
    if (!(q < t->body[ORC_MDF_M - 1])) return (uint64_t)(ORC_MDF_M - 1) << 20;
    int lo = 0, hi = ORC_MDF_M - 1;            /* body[lo] <= q < body[hi] */
    if (!(t->body[0] <= q)) return 0;
    while (hi - lo > 1) {
        int m = (lo + hi) / 2;
        if (t->body[m] <= q) lo = m; else hi = m;
    }
    return (uint64_t)lo << 20;
}

/* the grid point q_j = 2^(j/8 - 48) just below a tilt bound q_min:
 * j = floor(8 log2 q_min) + 384, at most 391; -1 below the grid */
static int grid_index(double qmin) {
    if (!(qmin >= exp2(-48.0))) return -1;
    int j = (int)floor(8.0 * log2(qmin)) + 384;
    return j > 391 ? 391 : j;
}

/* w0 for a tilt bound q_min: the table interval of its grid point */
static uint64_t word_floor_grid(const orc_mdf_table *t, double qmin) {
    int j = grid_index(qmin);
    return j < 0 ? 0 : word_floor(t, exp2(j / 8.0 - 48.0));
}

#define ORC_BAND_DJ 12        /* band B starts this many grid steps above q_min's grid point */
#define ORC_BAND_J2 351       /* and ends at the grid point q_J = 2^(-33/8) */

/* Band B's arc-measure bound, in units of pi: every tilt q in [q1, q2] (q2 <=
 * 1 - cos(pi / 2)) at every point of a segment with |k.N| in [lo, hi].  With a
 * = |k.N|, c_a = sqrt(1 - a^2) and b = c_a sin(theta), the window's two
 * intervals of cos(xi') are (S - a (1 - q)) / b and (-S - a (1 - q)) / b for S
 * in (S1, S2), each of width w <= (S2 - S1) / (c_a,min sin theta1).  The first
 * stays within |y| <= M = D / (c_a,min sin theta1) + hi tan(theta2 / 2) / c_a,min
 * (D = max |S - a| over the window and the segment; q / sin(theta) =
 * tan(theta / 2)), where the arcsine measure of an interval is at most its
 * width over sqrt(1 - M^2); the second lies beyond m = (S1 + lo (1 - q2)) /
 * sin theta2 (b <= sin theta2), so its measure is at most acos(m) (0 if m >= 1). */
static double band_b_bound(double lo, double hi, double S1, double S2, double q1, double q2) {
    double h = fmin(hi, 1.0);
    double camin = sqrt(fmax(0.0, 1.0 - h * h));
    double s1 = sqrt(q1 * (2.0 - q1)), s2 = sqrt(q2 * (2.0 - q2)), t2 = sqrt(q2 / (2.0 - q2));
    if (!(camin > 0.0) || !(s1 > 0.0)) return 1.0;
    double D = fmax(fabs(S1 - hi), fabs(S2 - lo));
    double M = D / (camin * s1) + hi * t2 / camin;
    double w = (S2 - S1) / (camin * s1);
    if (!(M < 1.0)) return 1.0;
    double same = w / sqrt(1.0 - M * M);
    double m = (S1 + lo * (1.0 - q2)) / s2;
    double mirror = m >= 1.0 ? 0.0 : acos(fmax(-1.0, m));
    return (same + mirror) / PI;
}

/* the bound of one order h on the segment with |k.N| in [lo, hi] */
static void bound_order(const geom *g, const orc_ray_consts *rc, int h, double lo, double hi, int band,
                        order_bound *b) {
    const orc_spec *s = g->s;
    memset(b, 0, sizeof *b);
    b->ra = 1.0;
    b->vstar = 1.0;
    b->pbar = 1.0;
    b->wspan = 1ull << 32;
    b->sA = 1.0;
    b->lam = rc->ord_qr[h];
    b->wn = b->wf = 1.0;
    b->psis = PI;
    b->pin = b->pio = 0.5;
    if (s->sampler == ORC_SAMPLER_THINNED && s->irc == ORC_IRC_NONE && rc->ord_qr[h] > 0) {
        /* the cone facing the ray (k.n of the sign of k.N): its crystallites are tilted
         * by at least the angle between a~0 and the grazing-angle range of the segment,
         * at least d, the distance between the sines; the other cone's by at least a~0.
         * The MDF decreases with the tilt, so W there bounds the cone on the segment:
         * rate Q cos a~0 2 pi (f(q_near) + f(q_far)) = ord_qr (wn + wf) / 2. */
        double a0 = rc->ord_alpha[h] + rc->shift_rad, s0 = sin(a0);
        double d = s0 < lo ? lo - s0 : (s0 > hi ? s0 - hi : 0.0);
        double hn = sin(0.5 * d), hf = sin(0.5 * a0);
        double q0 = 2.0 * hn * hn;
        b->wn = orc_mdf_W(s, q0) / g->W0;
        b->wf = orc_mdf_W(s, 2.0 * hf * hf) / g->W0;
        /* the window: q(psi) >= q0 + cos(a~0) cos(g_max) (1 - cos psi) >= q_v for |psi| >= psis */
        double sh = hi < 1.0 ? hi : 1.0, cmin = cos(a0) * sqrt(1.0 - sh * sh);
        if (q0 < g->none_qv && cmin > 0) {
            double xq = (g->none_qv - q0) / cmin;            /* 1 - cos(psis) */
            if (xq < 2.0) b->psis = 2.0 * asin(sqrt(0.5 * xq));
        }
        double fin = b->wn * (b->psis / PI), fout = b->psis < PI ? g->vstar * (1.0 - b->psis / PI) : 0.0;
        double tot = fin + fout + b->wf;
        b->lam = 0.5 * rc->ord_qr[h] * tot;
        b->pin = tot > 0 ? fin / tot : 1.0;
        b->pio = tot > 0 ? (fin + fout) / tot : 1.0;
        return;
    }
    if (s->sampler != ORC_SAMPLER_THINNED || s->irc == ORC_IRC_NONE || !(rc->ord_qr[h] > 0)) return;
    double aB = rc->ord_alpha[h] + rc->shift_rad;
    double xstar = g->xstar * rc->ord_w[h];          /* a curve w times as wide: X* scales by w */
    double sB = sin(aB);
    double d = sB < lo ? lo - sB : (sB > hi ? sB - hi : 0.0);
    double tmin = d - xstar;
    if (!(tmin > 0)) return;                          /* near Bragg: the plain stream */
    if (tmin > 0.5 * PI) tmin = 0.5 * PI;
    double sh = sin(0.5 * tmin);
    b->qmin = 2.0 * sh * sh;
    b->w0 = word_floor_grid(g->mdf, b->qmin);
    b->wspan = (1ull << 32) - b->w0;
    b->S1 = sin(fmax(0.0, aB - xstar));
    b->S2 = sin(fmin(0.5 * PI, aB + xstar));
    double bmin = sqrt(fmax(0.0, 1.0 - fmin(hi, 1.0) * fmin(hi, 1.0))) * sin(tmin);
    /* each of the two |k.n| windows spans w = (S2 - S1) / b in cos(xi'); an
     * interval of that width has arcsine measure at most acos(1 - w) / pi */
    double w = (b->S2 - b->S1) / bmin;
    b->pbar = (w >= 2.0 || !(bmin > 0)) ? 1.0 : fmin(1.0, 2.0 * acos(1.0 - w) / PI);
    b->w1 = b->w2 = b->w0;
    b->pbarB = b->pbar;
    int j0 = grid_index(b->qmin);
    if (band && j0 >= 0 && j0 + ORC_BAND_DJ < ORC_BAND_J2) {
        uint64_t w1 = word_floor(g->mdf, exp2((j0 + ORC_BAND_DJ) / 8.0 - 48.0));
        uint64_t w2 = word_floor(g->mdf, exp2(ORC_BAND_J2 / 8.0 - 48.0));
        if (w1 < w2) {
            /* tilts of band B: from the table knot that starts w1's interval to q_J */
            double pB = band_b_bound(lo, hi, b->S1, b->S2, g->mdf->body[w1 >> 20], exp2(ORC_BAND_J2 / 8.0 - 48.0));
            if (pB < b->pbar) {
                b->w1 = w1;
                b->w2 = w2;
                b->pbarB = pB;
            }
        }
    }
    double QR = rc->ord_qr[h];
    double PA = (double)((b->w1 - b->w0) + ((1ull << 32) - b->w2)) / 4294967296.0;
    double PB = (double)(b->w2 - b->w1) / 4294967296.0;
    double lA = PA * b->pbar, lB = PB * b->pbarB;
    b->sA = lA + lB > 0.0 ? lA / (lA + lB) : 1.0;
    double la = QR * g->vstar, lb = QR * (1.0 - g->vstar) * (lA + lB);
    b->vstar = g->vstar;
    b->lam = la + lb;
    b->ra = la / (la + lb);
}

static void bound_segment(const geom *g, const orc_ray_consts *rc, const double x[3], const double k[3],
                          seg_bound *b) {
    const orc_spec *s = g->s;
    memset(b, 0, sizeof *b);
    b->n = rc->n_orders;
    double lo = 0.0, hi = 1.0;
    if (s->sampler == ORC_SAMPLER_THINNED && !rc->no_bragg) {
        int face;
        double se = exit_distance(g, x, k, &face);
        double xe[3], N0[3], N1[3], t1[3], t2[3];
        for (int i = 0; i < 3; ++i) xe[i] = x[i] + se * k[i];
        local_frame(g, x, N0, t1, t2);
        local_frame(g, xe, N1, t1, t2);
        double k0 = dot3(k, N0), k1 = dot3(k, N1);
        lo = fmin(fabs(k0), fabs(k1));
        hi = fmax(fabs(k0), fabs(k1));
        if ((k0 < 0) != (k1 < 0)) lo = 0.0;         /* k.N is monotone along a line: it crossed 0 */
    }
    double lam = 0.0;
    for (int h = 0; h < b->n; ++h) {
        bound_order(g, rc, h, lo, hi, b->n == 1, &b->o[h]);
        lam += b->o[h].lam;
    }
    double run = 0.0;
    for (int h = 0; h < b->n; ++h) {
        run += b->o[h].lam;
        b->cum[h] = lam > 0 ? run / lam : 1.0;
    }
    b->cum[b->n - 1] = 1.0;
    b->mu = rc->mu0 + lam;
    b->pa = rc->mu0 / b->mu;
}

/* arc measure P_xi (in units of pi) of the azimuths xi' in [0, pi] with
 * |a + b cos xi'| in (S1, S2); the arcs themselves in arc[4] (start, length) */
static double azimuth_arcs(double a, double b, double S1, double S2, double arc[4]) {
    double iv[2][2] = {{(S1 - a) / b, (S2 - a) / b}, {(-S2 - a) / b, (-S1 - a) / b}};
    double tot = 0.0;
    for (int j = 0; j < 2; ++j) {
        double l = fmax(-1.0, iv[j][0]), h = fmin(1.0, iv[j][1]);
        arc[2 * j] = 0.0;
        arc[2 * j + 1] = 0.0;
        if (l < h) {
            arc[2 * j] = acos(h);
            arc[2 * j + 1] = acos(l) - acos(h);
            tot += arc[2 * j + 1];
        }
    }
    return tot / PI;
}

/* unit vectors perpendicular to k: e1 along the part of N perpendicular to k
 * (t1's part when k is along N), e2 = k x e1 */
static void cone_axes(const double k[3], const double N[3], const double t1[3], double e1[3], double e2[3]) {
    double kN = dot3(k, N);
    for (int i = 0; i < 3; ++i) e1[i] = N[i] - kN * k[i];
    if (normalize3(e1)) {
        double kt = dot3(k, t1);
        for (int i = 0; i < 3; ++i) e1[i] = t1[i] - kt * k[i];
        normalize3(e1);
    }
    cross3(k, e1, e2);
}

/* a scatter candidate of order h without rocking curve: the crystallite normal
 * n = sg sin(a~0) k + cos(a~0) (cos(psi) e1 + sin(psi) e2) on the cone
 * k.n = sg sin(a~0).  Plain: sg = -1 if the top bit of u2 is clear, +1 if set;
 * psi = 2 pi u3; P = f(n) G / f(0) = W(1 - n.N) G / W(0).  Thinned: by u2
 * against the shares pin, pio the facing cone's window (psi = psis (2 u3 - 1)),
 * the rest of the facing cone (psi = psis + 2 (pi - psis) u3) or the other cone
 * (psi = 2 pi u3); P = W(1 - n.N) G / (W(0) x that part's bound). */
static void cone_candidate(const geom *g, const orc_ray_consts *rc, int h, const order_bound *ob, const double x[3],
                           const double k[3], int pol, const double p[3], const uint32_t w[4], double ks[3],
                           double *P) {
    double N[3], t1[3], t2[3], e1[3], e2[3], n[3];
    local_frame(g, x, N, t1, t2);
    cone_axes(k, N, t1, e1, e2);
    double a0 = rc->ord_alpha[h] + rc->shift_rad, s0 = sin(a0), c0 = cos(a0);
    double sg, wb = 1.0;                             /* the cone, and the bound of W / W(0) on it */
    double psi = 2.0 * PI * U(w[3]);
    if (g->s->sampler == ORC_SAMPLER_THINNED) {
        /* the facing cone (k.n of the sign of k.N): its window or the rest; or the other cone */
        double kN = dot3(k, N), side = kN < 0 ? -1.0 : 1.0, u2 = U(w[2]), u3 = U(w[3]);
        if (u2 < ob->pin) {
            sg = side;
            wb = ob->wn;
            psi = ob->psis * (2.0 * u3 - 1.0);
        } else if (u2 < ob->pio) {
            sg = side;
            wb = g->vstar;
            psi = ob->psis + 2.0 * (PI - ob->psis) * u3;
        } else {
            sg = -side;
            wb = ob->wf;
        }
    } else {
        sg = (w[2] & 0x80000000u) ? 1.0 : -1.0;
    }
    for (int i = 0; i < 3; ++i) n[i] = sg * s0 * k[i] + c0 * (cos(psi) * e1[i] + sin(psi) * e2[i]);
    double q = 1.0 - dot3(n, N);                     /* 1 - cos(theta), the crystallite's tilt */
    for (int i = 0; i < 3; ++i) ks[i] = k[i] - 2.0 * (sg * s0) * n[i];   /* k.n = sg s0 */
    double G;
    if (pol) {
        double pk = dot3(p, ks);
        G = 1.0 - pk * pk;                           /* Eq. (G_pol) */
    } else {
        double c2 = cos(2.0 * a0);
        G = 0.5 * (1.0 + c2 * c2);                   /* Eq. (G_unpol) at a~0 */
    }
    *P = orc_mdf_W(g->s, q) / g->W0 / wb * G;
}

/* the depth walk of one ray from its entry point (Sec. 2.2.4) */
static void walk(const geom *g, const orc_ray_consts *rc, double x[3], double k[3], int pol, double p[3],
                 wsrc *ws, orc_record *rec) {
    const orc_spec *s = g->s;
    int nrefl = 0;
    int64_t ncoll = 0;
    int outcome = ORC_STUCK;
    seg_bound sb;
    bound_segment(g, rc, x, k, &sb);
    for (;;) {
        if (ncoll >= s->max_collisions) { outcome = ORC_STUCK; break; }
        uint32_t w[4];
        if (!next4(ws, w)) { outcome = ORC_STUCK; break; }
        double l = -log(U(w[0])) / sb.mu;              /* Eq. (AnyEvent) with the majorant */
        int face;
        double se = exit_distance(g, x, k, &face);
        if (l > se) {                                   /* leaves before the event */
            for (int i = 0; i < 3; ++i) x[i] += se * k[i];
            outcome = face;
            break;
        }
        for (int i = 0; i < 3; ++i) x[i] += l * k[i];
        ++ncoll;
        double u1 = U(w[1]);
        if (u1 < sb.pa) { outcome = ORC_ABSORBED; break; }
        double v = (u1 - sb.pa) / (1.0 - sb.pa);
        /* the reflection order, by its share of the candidate rate (superposition
         * over H); the conditional uniform stays the acceptance uniform */
        int h = 0;
        if (sb.n > 1) {
            while (h < sb.n - 1 && !(v < sb.cum[h])) ++h;
            double c0 = h > 0 ? sb.cum[h - 1] : 0.0;
            v = (v - c0) / (sb.cum[h] - c0);
        }
        double ks[3], P;                                 /* reflected direction, acceptance probability */
        if (g->irc_none) {
            cone_candidate(g, rc, h, &sb.o[h], x, k, pol, p, w, ks, &P);
            goto decide;
        }
        const order_bound *ob = &sb.o[h];
        double N[3], t1[3], t2[3];
        local_frame(g, x, N, t1, t2);
        double q, xi;
        if (v < ob->ra) {                                /* process (a), or the plain stream */
            v = ob->ra < 1.0 ? (v / ob->ra) * ob->vstar : v;
            q = orc_mdf_table_lookup(g->mdf, w[2]);
            xi = 2.0 * PI * U(w[3]);
        } else {                                         /* process (b) */
            double vb = (v - ob->ra) / (1.0 - ob->ra), pb;
            uint64_t wq;
            if (vb < ob->sA) {                           /* band A: words [w0, w1) and [w2, 2^32) */
                if (ob->sA < 1.0) vb /= ob->sA;
                uint64_t span = (ob->w1 - ob->w0) + ((1ull << 32) - ob->w2);
                wq = ob->w0 + (((uint64_t)w[2] * span) >> 32);
                if (wq >= ob->w1) wq += ob->w2 - ob->w1;
                pb = ob->pbar;
            } else {                                     /* band B: words [w1, w2) */
                vb = (vb - ob->sA) / (1.0 - ob->sA);
                wq = ob->w1 + (((uint64_t)w[2] * (ob->w2 - ob->w1)) >> 32);
                pb = ob->pbarB;
            }
            v = ob->vstar + (1.0 - ob->vstar) * vb;
            q = orc_mdf_table_lookup(g->mdf, (uint32_t)wq);
            if (q < ob->qmin || q > 2.0 - ob->qmin) continue;  /* cannot reflect */
            double kN = dot3(k, N), sa_ = fabs(kN), ca_ = sqrt(fmax(0.0, 1.0 - kN * kN));
            double a = (kN < 0 ? -sa_ : sa_) * (1.0 - q), b = ca_ * sqrt(q * (2.0 - q));
            double arc[4];
            double Pxi = azimuth_arcs(a, b, ob->S1, ob->S2, arc);
            double t3 = U(w[3]);
            if (!(t3 * pb < Pxi)) continue;                 /* outside the arcs: cannot reflect */
            double L = arc[1] + arc[3];
            double pos = (t3 * pb / Pxi) * 2.0 * L, sgn = 1.0;
            if (pos >= L) { pos -= L; sgn = -1.0; }
            double xp = pos < arc[1] ? arc[0] + pos : arc[2] + (pos - arc[1]);
            xi = atan2(dot3(k, t2), dot3(k, t1)) + sgn * xp;
        }
        double ct = 1.0 - q, st = sqrt(q * (2.0 - q));
        double cx = cos(xi), sx = sin(xi);
        double n[3];
        for (int i = 0; i < 3; ++i) n[i] = ct * N[i] + st * (cx * t1[i] + sx * t2[i]);
        double kn = dot3(k, n);
        double sa = fabs(kn);
        if (sa > 1.0) sa = 1.0;
        double at = asin(sa);                            /* incidence on the crystallite */
        double delta = at - rc->ord_alpha[h] - rc->shift_rad;
        for (int i = 0; i < 3; ++i) ks[i] = k[i] - 2.0 * kn * n[i];   /* reflection equation */
        double G;
        if (pol) {
            double pk = dot3(p, ks);
            G = 1.0 - pk * pk;                           /* G = 1 - (p . k_s)^2, Eq. (G_pol) */
        } else {
            double c2 = cos(2.0 * at);
            G = 0.5 * (1.0 + c2 * c2);                   /* Eq. (G_unpol) */
        }
        /* the order's curve is the described one w_h times as wide: R_h / R_h,max = R(x / w_h) / R_max */
        P = irc_eval(&g->irc, delta / rc->ord_w[h]) * G / g->irc_max;
    decide:
        if (v < P) {
            ++nrefl;
            if (nrefl > s->max_reflections) { outcome = ORC_CAPPED; break; }
            memcpy(k, ks, sizeof ks);
            normalize3(k);
            if (pol) {                                   /* p_s = (p - (p.k_s) k_s) / sqrt(1 - (p.k_s)^2) */
                double pk = dot3(p, k);
                double d = sqrt(1.0 - pk * pk);
                for (int i = 0; i < 3; ++i) p[i] = (p[i] - pk * k[i]) / d;
                normalize3(p);
            }
            bound_segment(g, rc, x, k, &sb);             /* a new straight segment */
        }
    }
    rec->outcome = outcome;
    rec->nrefl = nrefl;
    rec->ncoll = ncoll;
    memcpy(rec->pos, x, 3 * sizeof(double));
    memcpy(rec->dir, k, 3 * sizeof(double));
    for (int i = 0; i < 3; ++i) rec->pol[i] = pol ? p[i] : 0.0;
    rec->u_mm = NAN; rec->v_mm = NAN; rec->ix = -1; rec->iy = -1; rec->det_hit = 0;
    if (outcome == ORC_EXIT_FRONT || outcome == ORC_EXIT_BACK || outcome == ORC_EXIT_SIDE)
        detector(g, x, k, rec);
}

/* polarisation of a ray: p0 projected perpendicular to k, or none */
static int project_pol(const double p0[3], const double k[3], double p[3]) {
    double pk = dot3(p0, k);
    for (int i = 0; i < 3; ++i) p[i] = p0[i] - pk * k[i];
    double n = sqrt(dot3(p, p));
    if (!(n > 1e-12)) { p[0] = p[1] = p[2] = 0.0; return 0; }
    for (int i = 0; i < 3; ++i) p[i] /= n;
    return 1;
}

/* ------------------------------------------------------------------ */
/* source (Sec. 2.1)                                                   */
/* ------------------------------------------------------------------ */
static void source_basis(const double a[3], double b1[3], double b2[3]) {
    int j = 0;
    if (fabs(a[1]) < fabs(a[j])) j = 1;
    if (fabs(a[2]) < fabs(a[j])) j = 2;
    double e[3] = {0, 0, 0};
    e[j] = 1.0;
    cross3(e, a, b1);
    normalize3(b1);
    cross3(a, b1, b2);
}

/* Sec. 2.1 draws the source's energy, direction and spot position from
 * independent uniforms; which Philox word feeds which draw is a convention.
 * Here a is the ray's first block (call 0): spot radius and angle, 1 - cos(phi)
 * and the azimuth, i.e. all that the crystal-entry test needs; b is its second
 * block (call 1): the component, its parameter and the Gaussian line's pair. */
static void sample_source(const orc_source *src, const double cumw[], const double *tcdf,
                          const double ax[3], const double b1[3], const double b2[3], const uint32_t a[4],
                          const uint32_t b[4], double *E, double o[3], double k[3]) {
    /* energy (second block): component by cumulative weight, then its parameter */
    double uc = U(b[0]);
    int c = src->n_comp - 1;
    for (int i = 0; i < src->n_comp; ++i)
        if (uc < cumw[i]) { c = i; break; }
    const orc_component *cp = &src->comp[c];
    double up = U(b[1]);
    switch (cp->kind) {
    case ORC_SRC_MONO: *E = cp->e0_keV; break;
    case ORC_SRC_GAUSS: {
        double z = sqrt(-2.0 * log(U(b[2]))) * cos(2.0 * PI * U(b[3]));
        *E = cp->e0_keV + cp->width_keV * z;
        break;
    }
    case ORC_SRC_LORENTZ: {                  /* Cauchy truncated to E > 0 */
        double gam = 0.5 * cp->width_keV;
        double F0 = 0.5 + atan(-cp->e0_keV / gam) / PI;
        double uu = F0 + up * (1.0 - F0);
        *E = cp->e0_keV + gam * tan(PI * (uu - 0.5));
        break;
    }
    case ORC_SRC_INV_E: *E = cp->lo_keV * pow(cp->hi_keV / cp->lo_keV, up); break;
    case ORC_SRC_UNIFORM: *E = cp->lo_keV + (cp->hi_keV - cp->lo_keV) * up; break;
    case ORC_SRC_TABLE: {                    /* inverse of the piecewise-linear CDF */
        int i = 0;
        while (!(up < tcdf[i + 1])) ++i;      /* the interval with C_i <= up < C_i+1 */
        const double *x = src->table_keV;
        *E = x[i] + (up - tcdf[i]) / (tcdf[i + 1] - tcdf[i]) * (x[i + 1] - x[i]);
        break;
    }
    default: *E = NAN;
    }
    /* direction (first block): uniform in solid angle inside the cone */
    double hs = sin(0.5 * src->cone_half_angle_rad);
    double w = U(a[2]) * 2.0 * hs * hs;          /* 1 - cos(phi) */
    double cphi = 1.0 - w, sphi = sqrt(w * (2.0 - w));
    double beta = 2.0 * PI * U(a[3]);
    double cb = cos(beta), sb = sin(beta);
    for (int i = 0; i < 3; ++i) k[i] = cphi * ax[i] + sphi * (cb * b1[i] + sb * b2[i]);
    /* origin (first block): 2-D Gaussian spot in the plane perpendicular to the cone axis */
    double r = sqrt(-2.0 * log(U(a[0])));
    double ang = 2.0 * PI * U(a[1]);
    double z1 = r * cos(ang), z2 = r * sin(ang);
    double s1 = src->spot_fwhm_mm[0] / (2.0 * sqrt(2.0 * LN2));
    double s2 = src->spot_fwhm_mm[1] / (2.0 * sqrt(2.0 * LN2));
    for (int i = 0; i < 3; ++i) o[i] = src->origin[i] + s1 * z1 * b1[i] + s2 * z2 * b2[i];
}

typedef struct {
    const geom *g;
    const orc_source *src;
    const double *cumw;
    const double *tcdf;      /* CDF of the tabulated spectrum at its knots, or NULL */
    double ax[3], b1[3], b2[3];
    uint64_t begin, end, offset;
    uint32_t key[2];
    int64_t *image;          /* private per thread */
    int64_t *eimage;         /* private per thread, or NULL */
    const orc_qe *qe;
    const orc_rays *rays;    /* user-supplied rays, or NULL (sampled source) */
    orc_tally tally;
    orc_record *records;
} job;

static void trace_one(job *J, uint64_t i) {
    const geom *g = J->g;
    const orc_spec *s = g->s;
    uint64_t ray = J->offset + i;
    wsrc ws = {0};
    ws.key[0] = J->key[0]; ws.key[1] = J->key[1];
    ws.ray = ray; ws.call = 0;
    double E, o[3], k[3], p[3], pv[3] = {0, 0, 0};
    int pol = 0;
    if (J->rays) {
        const orc_rays *R = J->rays;
        E = R->E[i];
        o[0] = R->ox[i]; o[1] = R->oy[i]; o[2] = R->oz[i];
        k[0] = R->kx[i]; k[1] = R->ky[i]; k[2] = R->kz[i];
        if (normalize3(k)) E = NAN;                     /* a zero direction cannot enter */
        if (R->px) {
            double p0[3] = {R->px[i], R->py[i], R->pz[i]};
            pol = project_pol(p0, k, pv);
        }
        ws.call = 2;                                    /* the walk's words, as for sampled rays */
    } else {
        uint32_t a[4], b[4];
        next4(&ws, a);
        next4(&ws, b);
        sample_source(J->src, J->cumw, J->tcdf, J->ax, J->b1, J->b2, a, b, &E, o, k);
        pol = project_pol(J->src->polarization, k, pv);
    }
    orc_record rec;
    memset(&rec, 0, sizeof rec);
    rec.ray_id = ray;
    rec.energy_keV = E;
    J->tally.emitted++;
    int hit = (E > 0 && isfinite(E)) ? entry(g, o, k, p) : 0;
    if (!hit) {
        J->tally.miss++;
        rec.outcome = ORC_MISS;
        memcpy(rec.pos, o, sizeof rec.pos);
        memcpy(rec.dir, k, sizeof rec.dir);
        for (int c = 0; c < 3; ++c) rec.pol[c] = pol ? pv[c] : 0.0;
        rec.u_mm = NAN; rec.v_mm = NAN; rec.ix = -1; rec.iy = -1;
    } else {
        orc_ray_consts rc;
        ray_constants(s, E, g->none_fac, &rc);
        if (rc.no_bragg) J->tally.no_bragg++;
        rec.no_bragg = rc.no_bragg;
        walk(g, &rc, p, k, pol, pv, &ws, &rec);
        J->tally.collisions += (uint64_t)rec.ncoll;
        J->tally.refl_hist[rec.nrefl < 15 ? rec.nrefl : 15]++;
        switch (rec.outcome) {
        case ORC_ABSORBED: J->tally.absorbed++; break;
        case ORC_EXIT_FRONT: J->tally.exit_front++; break;
        case ORC_EXIT_BACK: J->tally.exit_back++; break;
        case ORC_EXIT_SIDE: J->tally.exit_side++; break;
        case ORC_CAPPED: J->tally.capped++; break;
        case ORC_STUCK: J->tally.stuck++; break;
        }
        if (rec.det_hit) {
            J->tally.det_hits++;
            J->image[(int64_t)rec.iy * s->det_nx + rec.ix] += 1;
            if (J->eimage)
                J->eimage[(int64_t)rec.iy * s->det_nx + rec.ix] += (int64_t)llround(E * orc_qe_eval(J->qe, E) * 1e6);
        }
    }
    if (J->records) J->records[i] = rec;
}

static void *thread_main(void *arg) {
    job *J = (job *)arg;
    for (uint64_t i = J->begin; i < J->end; ++i) trace_one(J, i);
    return NULL;
}

double orc_qe_eval(const orc_qe *q, double E) {
    if (!q || q->n <= 0) return 1.0;
    if (E <= q->keV[0]) return q->qe[0];
    for (int i = 1; i < q->n; ++i)
        if (E <= q->keV[i]) {
            double f = (E - q->keV[i - 1]) / (q->keV[i] - q->keV[i - 1]);
            return q->qe[i - 1] + f * (q->qe[i] - q->qe[i - 1]);
        }
    return q->qe[q->n - 1];
}

int orc_trace(const orc_spec *s, const orc_source *src, uint64_t n_rays, uint64_t seed,
              uint64_t ray_offset, int n_threads, int64_t *image, orc_tally *tally,
              orc_record *records) {
    return orc_trace_energy(s, src, n_rays, seed, ray_offset, n_threads, image, NULL, NULL, tally, records);
}

static int trace_driver(const orc_spec *s, const orc_source *src, const orc_rays *rays, uint64_t n_rays,
                        uint64_t seed, uint64_t ray_offset, int n_threads, int64_t *image,
                        int64_t *energy_image, const orc_qe *qe, orc_tally *tally, orc_record *records);

/* CDF of a tabulated spectrum at its knots: C_0 = 0, C_i+1 = C_i + (p_i + p_i+1)/2 (x_i+1 - x_i),
 * divided by the total (the trapezoid rule; the CDF is linear between knots) */
static int build_table_cdf(const orc_source *src, double **out) {
    int n = src->n_table;
    if (!src->table_keV || !src->table_pdf || n < 2 || n > ORC_MAX_TABLE) return fail("bad spectrum table");
    for (int i = 0; i < n; ++i) {
        if (!isfinite(src->table_keV[i]) || !isfinite(src->table_pdf[i]) || src->table_pdf[i] < 0.0)
            return fail("bad spectrum table value");
        if (i > 0 && !(src->table_keV[i] > src->table_keV[i - 1])) return fail("spectrum knots not ascending");
    }
    if (!(src->table_keV[0] > 0.0)) return fail("spectrum energies must be positive");
    double *c = (double *)malloc((size_t)n * sizeof(double));
    if (!c) return fail("out of memory");
    double run = 0.0;
    c[0] = 0.0;
    for (int i = 0; i + 1 < n; ++i) {
        run += 0.5 * (src->table_pdf[i] + src->table_pdf[i + 1]) * (src->table_keV[i + 1] - src->table_keV[i]);
        c[i + 1] = run;
    }
    if (!(run > 0.0) || !isfinite(run)) { free(c); return fail("spectrum table has no mass"); }
    for (int i = 1; i < n; ++i) c[i] /= run;
    c[n - 1] = 1.0;
    *out = c;
    return 0;
}

int orc_trace_energy(const orc_spec *s, const orc_source *src, uint64_t n_rays, uint64_t seed,
                     uint64_t ray_offset, int n_threads, int64_t *image, int64_t *energy_image,
                     const orc_qe *qe, orc_tally *tally, orc_record *records) {
    if (!src) return fail("null argument");
    return trace_driver(s, src, NULL, n_rays, seed, ray_offset, n_threads, image, energy_image, qe, tally,
                        records);
}

int orc_trace_rays(const orc_spec *s, const orc_rays *rays, uint64_t n_rays, uint64_t seed,
                   uint64_t ray_offset, int n_threads, int64_t *image, int64_t *energy_image,
                   const orc_qe *qe, orc_tally *tally, orc_record *records) {
    if (!rays || !rays->ox || !rays->oy || !rays->oz || !rays->kx || !rays->ky || !rays->kz || !rays->E)
        return fail("null ray array");
    if (rays->px && (!rays->py || !rays->pz)) return fail("partial polarisation arrays");
    return trace_driver(s, NULL, rays, n_rays, seed, ray_offset, n_threads, image, energy_image, qe, tally,
                        records);
}

static int trace_driver(const orc_spec *s, const orc_source *src, const orc_rays *rays, uint64_t n_rays,
                        uint64_t seed, uint64_t ray_offset, int n_threads, int64_t *image,
                        int64_t *energy_image, const orc_qe *qe, orc_tally *tally, orc_record *records) {
    if (!s || !image || !tally) return fail("null argument");
    if (qe && (qe->n < 0 || qe->n > ORC_MAX_QE)) return fail("bad QE table");
    if (src && (src->n_comp < 1 || src->n_comp > ORC_MAX_COMP)) return fail("bad component count");
    geom g;
    if (geom_init(&g, s)) return -1;
    orc_mdf_table *tab = (orc_mdf_table *)malloc(sizeof(orc_mdf_table));
    if (!tab) return fail("out of memory");
    if (orc_mdf_build_table(s, tab)) { free(tab); return -1; }
    g.mdf = tab;
    double cumw[ORC_MAX_COMP], tot = 0.0;
    double ax[3] = {0, 0, 1}, b1[3] = {1, 0, 0}, b2[3] = {0, 1, 0};
    if (src) {
        for (int i = 0; i < src->n_comp; ++i) tot += src->comp[i].weight;
        double run = 0.0;
        for (int i = 0; i < src->n_comp; ++i) { run += src->comp[i].weight; cumw[i] = run / tot; }
        memcpy(ax, src->axis, sizeof ax);
        if (normalize3(ax)) { free(tab); return fail("bad source axis"); }
        source_basis(ax, b1, b2);
    }
    double *tcdf = NULL;
    if (src) {
        int uses = 0;
        for (int i = 0; i < src->n_comp; ++i) uses |= src->comp[i].kind == ORC_SRC_TABLE;
        if (uses && build_table_cdf(src, &tcdf)) { free(tab); return -1; }
    }

    if (n_threads <= 0) n_threads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (n_threads < 1) n_threads = 1;
    if ((uint64_t)n_threads > n_rays && n_rays > 0) n_threads = (int)n_rays;
    if (n_rays == 0) n_threads = 1;
    size_t npix = (size_t)s->det_nx * (size_t)s->det_ny;
    job *jobs = (job *)calloc((size_t)n_threads, sizeof(job));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) { free(tab); free(tcdf); free(jobs); free(th); return fail("out of memory"); }
    for (int t = 0; t < n_threads; ++t) {
        job *J = &jobs[t];
        J->g = &g; J->src = src; J->cumw = cumw; J->tcdf = tcdf;
        memcpy(J->ax, ax, sizeof ax); memcpy(J->b1, b1, sizeof b1); memcpy(J->b2, b2, sizeof b2);
        J->begin = n_rays * (uint64_t)t / (uint64_t)n_threads;
        J->end = n_rays * (uint64_t)(t + 1) / (uint64_t)n_threads;
        J->offset = ray_offset;
        J->key[0] = (uint32_t)seed; J->key[1] = (uint32_t)(seed >> 32);
        J->image = (t == 0) ? image : (int64_t *)calloc(npix, sizeof(int64_t));
        J->eimage = (!energy_image) ? NULL : (t == 0) ? energy_image : (int64_t *)calloc(npix, sizeof(int64_t));
        J->qe = qe;
        J->rays = rays;
        J->records = records;
        if (!J->image || (energy_image && !J->eimage)) { n_threads = t; break; }
    }
    int nt = n_threads;
    for (int t = 1; t < nt; ++t) pthread_create(&th[t], NULL, thread_main, &jobs[t]);
    if (nt > 0) thread_main(&jobs[0]);
    for (int t = 1; t < nt; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nt; ++t) {
        orc_tally *a = &jobs[t].tally;
        tally->emitted += a->emitted; tally->miss += a->miss; tally->absorbed += a->absorbed;
        tally->exit_front += a->exit_front; tally->exit_back += a->exit_back;
        tally->exit_side += a->exit_side; tally->capped += a->capped; tally->stuck += a->stuck;
        tally->no_bragg += a->no_bragg; tally->det_hits += a->det_hits;
        tally->collisions += a->collisions;
        for (int h = 0; h < 16; ++h) tally->refl_hist[h] += a->refl_hist[h];
        if (t > 0) {
            for (size_t p = 0; p < npix; ++p) image[p] += jobs[t].image[p];
            free(jobs[t].image);
            if (energy_image) {
                for (size_t p = 0; p < npix; ++p) energy_image[p] += jobs[t].eimage[p];
                free(jobs[t].eimage);
            }
        }
    }
    free(jobs); free(th); free(tab); free(tcdf);
    return 0;
}

int orc_walk_injected_n(const orc_spec *s, int64_t n, const double *E, const double *pos, const double *dir,
                        const double *pol, const uint32_t *words, int64_t words_per_ray, orc_record *rec) {
    geom g;
    if (geom_init(&g, s)) return -1;
    orc_mdf_table *tab = (orc_mdf_table *)malloc(sizeof(orc_mdf_table));
    if (!tab) return fail("out of memory");
    if (orc_mdf_build_table(s, tab)) { free(tab); return -1; }
    g.mdf = tab;
    for (int64_t i = 0; i < n; ++i) {
        orc_ray_consts rc;
        ray_constants(s, E[i], g.none_fac, &rc);
        wsrc ws = {0};
        ws.words = words + i * words_per_ray; ws.n = words_per_ray; ws.pos = 0;
        double x[3], k[3];
        memcpy(x, pos + 3 * i, sizeof x);
        memcpy(k, dir + 3 * i, sizeof k);
        orc_record *r = rec + i;
        memset(r, 0, sizeof *r);
        r->energy_keV = E[i];
        r->no_bragg = rc.no_bragg;
        double pv[3] = {0, 0, 0};
        int pl = pol ? project_pol(pol + 3 * i, k, pv) : 0;
        walk(&g, &rc, x, k, pl, pv, &ws, r);
    }
    free(tab);
    return 0;
}

int orc_walk_injected(const orc_spec *s, double E, const double pos[3], const double dir[3],
                      const double *pol, const uint32_t *words, int64_t n_words, orc_record *rec) {
    return orc_walk_injected_n(s, 1, &E, pos, dir, pol, words, n_words, rec);
}

/* the thinned sampler's bounds of straight segments, for tests of its exactness */
int orc_segment_bounds(const orc_spec *s, int64_t n, const double *E, const double *xs, const double *ks, int h,
                       orc_seg_info *outs) {
    geom g;
    if (geom_init(&g, s)) return -1;
    orc_mdf_table *tab = (orc_mdf_table *)malloc(sizeof(orc_mdf_table));
    if (!tab) return fail("out of memory");
    if (orc_mdf_build_table(s, tab)) { free(tab); return -1; }
    g.mdf = tab;
    for (int64_t i = 0; i < n; ++i) {
        const double *x = xs + 3 * i, *k = ks + 3 * i;
        orc_seg_info *out = outs + i;
        memset(out, 0, sizeof *out);
        orc_ray_consts rc;
        ray_constants(s, E[i], g.none_fac, &rc);
        if (h < 0 || h >= rc.n_orders) { free(tab); return fail("order out of range"); }
        int face;
        out->s_exit = exit_distance(&g, x, k, &face);
        out->face = face;
        double xe[3], N0[3], N1[3], t1[3], t2[3];
        for (int j = 0; j < 3; ++j) xe[j] = x[j] + out->s_exit * k[j];
        local_frame(&g, x, N0, t1, t2);
        local_frame(&g, xe, N1, t1, t2);
        out->kN0 = dot3(k, N0);
        out->kN1 = dot3(k, N1);
        seg_bound sb;
        bound_segment(&g, &rc, x, k, &sb);
        const order_bound *b = &sb.o[h];
        out->xstar = g.xstar * rc.ord_w[h];
        out->vstar = g.vstar;
        out->irc_max = g.irc_max;
        out->W0 = g.W0;
        out->none_qv = g.none_qv;
        out->alpha0 = rc.ord_alpha[h] + rc.shift_rad;
        out->thinned = b->ra < 1.0 || (g.irc_none && s->sampler == ORC_SAMPLER_THINNED && rc.ord_qr[h] > 0);
        out->ra = b->ra;
        out->qmin = b->qmin;
        out->pbar = b->pbar;
        out->S1 = b->S1;
        out->S2 = b->S2;
        out->w0 = b->w0;
        out->wspan = b->wspan;
        out->w1 = b->w1;
        out->w2 = b->w2;
        out->pbarB = b->pbarB;
        out->sA = b->sA;
        out->lam = b->lam;
        out->mu = sb.mu;
        out->pa = sb.pa;
        out->wn = b->wn;
        out->wf = b->wf;
        out->psis = b->psis;
        out->pin = b->pin;
        out->pio = b->pio;
    }
    free(tab);
    return 0;
}

/* ------------------------------------------------------------------ */
/* accepted crystallites at fixed incidence (flat frame N = z, k in x-z) */
/* ------------------------------------------------------------------ */
int64_t orc_sample_crystallites(const orc_spec *s, double E, double alpha, int64_t n,
                                uint64_t seed, double *delta_out, double *psi_out) {
    if (s->irc == ORC_IRC_NONE) return fail("no rocking curve: every accepted Delta is 0");
    orc_mdf_table *tab = (orc_mdf_table *)malloc(sizeof(orc_mdf_table));
    if (!tab) return fail("out of memory");
    if (orc_mdf_build_table(s, tab)) { free(tab); return -1; }
    orc_ray_consts rc;
    orc_ray_constants(s, E, &rc);
    irc_params ip;
    irc_prepare(s, &ip);
    double irc_max = irc_eval(&ip, 0.0);
    double N[3] = {0, 0, 1}, t1[3] = {1, 0, 0}, t2[3] = {0, 1, 0};
    double k[3] = {cos(alpha), 0.0, -sin(alpha)};
    /* psi is measured about k from the part of N perpendicular to k */
    double e1[3], e2[3], kN = dot3(k, N);
    for (int i = 0; i < 3; ++i) e1[i] = N[i] - kN * k[i];
    normalize3(e1);
    cross3(k, e1, e2);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t got = 0;
    for (uint64_t it = 0; got < n && it < (uint64_t)4e10; ++it) {
        uint32_t ctr[4] = {(uint32_t)it, (uint32_t)(it >> 32), 0u, 1u}, w[4];
        orc_philox4x32_10(ctr, key, w);
        double q = orc_mdf_table_lookup(tab, w[2]);
        double ct = 1.0 - q, st = sqrt(q * (2.0 - q));
        double xi = 2.0 * PI * U(w[3]);
        double nn[3];
        for (int i = 0; i < 3; ++i) nn[i] = ct * N[i] + st * (cos(xi) * t1[i] + sin(xi) * t2[i]);
        double kn = dot3(k, nn);
        double sa = fabs(kn);
        if (sa > 1) sa = 1;
        double at = asin(sa);
        double delta = at - rc.alpha_B - rc.shift_rad;
        double c2 = cos(2.0 * at);
        double P = irc_eval(&ip, delta / rc.ord_w[0]) * 0.5 * (1.0 + c2 * c2) / irc_max;   /* the first order */
        if (U(w[1]) < P) {
            double sgn = kn < 0 ? 1.0 : -1.0;   /* H or H-bar: the normal facing the ray */
            double np[3];
            for (int i = 0; i < 3; ++i) np[i] = sgn * nn[i] - (sgn * kn) * k[i];
            delta_out[got] = delta;
            psi_out[got] = atan2(dot3(np, e2), dot3(np, e1));
            ++got;
        }
    }
    free(tab);
    return got;
}

/* ------------------------------------------------------------------ */
/* reflection rate r(alpha) by quadrature of Eq. (ReflXsection)        */
/*   r = Q int dDelta R(Delta) cos(a~) G(a~) int dpsi f(theta(alpha,psi,a~)) */
/* with f the MDF normalised on the sphere and theta from Eq. (ThetaPsi), */
/* written as 1 - cos(theta) = 2 sin^2((alpha-a~)/2) + 2 cos(alpha) cos(a~) sin^2(psi/2). */
/* ------------------------------------------------------------------ */
typedef struct { const orc_spec *s; double alpha, at, Z, aB, shift, w; irc_params irc; } rr_ctx;

static double rr_inner(const void *vp, double psi) {
    const rr_ctx *c = (const rr_ctx *)vp;
    double h1 = sin(0.5 * (c->alpha - c->at)), h2 = sin(0.5 * psi);
    double q = 2.0 * h1 * h1 + 2.0 * cos(c->alpha) * cos(c->at) * h2 * h2;
    if (q > orc_mdf_qmax(c->s)) return 0.0;
    return orc_mdf_W(c->s, q) / (2.0 * PI * c->Z);
}
static double rr_psi_integral(rr_ctx *c) {
    /* 2 * int_0^pi, on geometric panels in psi (narrow peak at psi = 0) */
    double sum = 0.0, a = 0.0, b = 1e-9;
    while (a < PI) {
        if (b > PI) b = PI;
        sum += integrate(rr_inner, c, a, b, 1e-11);
        a = b; b *= 1.5;
    }
    return 2.0 * sum;
}
static double rr_outer(const void *vp, double x) {
    rr_ctx *c = (rr_ctx *)vp;
    double at = c->aB + c->shift + x;
    if (at < 0 || at > 0.5 * PI) return 0.0;
    c->at = at;
    double c2 = cos(2.0 * at);
    double G = 0.5 * (1.0 + c2 * c2);
    double R = irc_eval(&c->irc, x / c->w) / c->w;       /* the order's curve: w times as wide, unit area */
    if (R == 0) return 0.0;
    return R * cos(at) * G * rr_psi_integral(c);
}
double orc_reflection_rate(const orc_spec *s, double E, double alpha) {
    orc_ray_consts rc;
    orc_ray_constants(s, E, &rc);
    if (rc.no_bragg) return 0.0;
    /* the sum over the reflection orders H of the paper's cross-section */
    double total = 0.0;
    double Z = orc_mdf_norm(s);
    for (int h = 0; h < rc.n_orders; ++h) {
        if (!(rc.ord_Q[h] > 0)) continue;
        rr_ctx c = {s, alpha, 0.0, Z, rc.ord_alpha[h], rc.shift_rad, rc.ord_w[h], {0}};
        irc_prepare(s, &c.irc);
        if (s->irc == ORC_IRC_NONE) {
            /* R = delta(Delta): the outer integral is its integrand at Delta = 0 */
            double at = rc.ord_alpha[h] + rc.shift_rad;
            if (!(at > 0 && at < 0.5 * PI)) continue;
            c.at = at;
            double c2 = cos(2.0 * at);
            total += rc.ord_Q[h] * cos(at) * 0.5 * (1.0 + c2 * c2) * rr_psi_integral(&c);
            continue;
        }
        double lo = -(rc.ord_alpha[h] + rc.shift_rad), hi = 0.5 * PI - rc.ord_alpha[h] - rc.shift_rad;
        /* geometric panels in |x| on each side of the IRC centre */
        double w = (s->irc_fwhm_rad > 0 ? s->irc_fwhm_rad : 1e-5) * rc.ord_w[h];
        double sum = 0.0;
        for (int side = 0; side < 2; ++side) {
            double lim = side ? hi : -lo;
            double a = 0.0, b = 1e-3 * w;
            while (a < lim) {
                if (b > lim) b = lim;
                double pa = side ? a : -b, pb = side ? b : -a;
                sum += integrate(rr_outer, &c, pa, pb, 1e-9);
                a = b; b *= 2.0;
            }
        }
        total += rc.ord_Q[h] * sum;
    }
    return total;
}
