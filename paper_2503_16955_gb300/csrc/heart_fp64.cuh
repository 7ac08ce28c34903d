// heart_fp64.cuh -- device functions of the plain FP64 ray path: one ray per
// thread, every quantity in double precision, positions in the global frame.
// This is the reference-precision GPU path that replays the CPU oracle's
// random streams ray by ray (same Philox words, same decisions).
#pragma once
#include <stdint.h>

#include "heart_internal.h"

namespace heart {

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
    // Salmon et al. (SC'11) Philox4x32 with 10 rounds: two 32x32->64
    // multiplies per round, Weyl-sequence key schedule.
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

__device__ __forceinline__ double u01_64(uint32_t w) {
    return ((double)w + 0.5) * 2.3283064365386962890625e-10;   // (w + 1/2) 2^-32
}

__device__ __forceinline__ double dot3d(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

struct RayOut64 {
    int outcome, nrefl, ix, iy, det_hit, no_bragg;
    long long ncoll;
    double E, pos[3], dir[3], u, v, pol[3];
};

// polarisation of a ray: p0 projected perpendicular to k, or none
__device__ __forceinline__ int project_pol64(const double p0[3], const double k[3], double p[3]) {
    const double pk = dot3d(p0, k);
    for (int i = 0; i < 3; ++i) p[i] = p0[i] - pk * k[i];
    const double n = sqrt(dot3d(p, p));
    if (!(n > 1e-12)) { p[0] = p[1] = p[2] = 0.0; return 0; }
    for (int i = 0; i < 3; ++i) p[i] /= n;
    return 1;
}

// mosaic quantile q = 1 - cos(theta) from one 32-bit word (table in smem)
__device__ __forceinline__ double mdf_q64(const double *tab, uint32_t w) {
    const uint32_t i = w >> 20;
    if (i < (uint32_t)(kMdfM - 1)) {
        const double f = ((double)(w & 0xFFFFFu) + 0.5) * (1.0 / 1048576.0);
        const double a = tab[i], b = tab[i + 1];
        return a + f * (b - a);
    }
    const double m = (double)(0xFFFFFFFFu - w) + 0.5;
    const double y = (32.0 - log2(m) - 12.0) * (kMdfT / 21.0);
    int j = (int)floor(y);
    j = j < 0 ? 0 : (j > kMdfT - 1 ? kMdfT - 1 : j);
    const double f = y - j;
    const double a = tab[kMdfM + j], b = tab[kMdfM + j + 1];
    return a + f * (b - a);
}

__host__ __device__ __forceinline__ double dp_reflectivity64(double y, double g) {
    const double ar = y * y - g * g - 1.0, ai = 2.0 * y * g;
    const double r = hypot(ar, ai);
    double zr, zi;
    if (ar >= 0) { zr = sqrt(0.5 * (r + ar)); zi = (zr > 0) ? 0.5 * ai / zr : 0.0; }
    else { zi = copysign(sqrt(0.5 * (r - ar)), ai); zr = 0.5 * ai / zi; }
    const double m1 = hypot(y - zr, g - zi), m2 = hypot(y + zr, g + zi);
    const double m = m1 > m2 ? m1 : m2;
    return 1.0 / (m * m);
}

// unit-area rocking curve at x = Delta - Delta_M
__host__ __device__ __forceinline__ double irc64(const SpecParams &S, double x) {
    switch (S.irc) {
    case HEART_IRC_DARWIN: {
        const double y = fabs(x) / S.irc_delta;
        if (y <= 1.0) return 1.0 / S.irc_norm;
        const double d = y + sqrt(y * y - 1.0);
        return 1.0 / (d * d * S.irc_norm);
    }
    case HEART_IRC_DARWIN_PRINS: return dp_reflectivity64(x / S.irc_delta, S.irc_g) / S.irc_norm;
    case HEART_IRC_PSEUDO_VOIGT: {
        const double F = S.irc_fwhm;
        const double L = F / (2.0 * 3.14159265358979323846) / (0.25 * F * F + x * x);
        const double c = 2.772588722239781 / (F * F);            // 4 ln 2 / F^2
        const double G = sqrt(c / 3.14159265358979323846) * exp(-c * x * x);
        return S.irc_eta * L + (1.0 - S.irc_eta) * G;
    }
    case HEART_IRC_GAUSSIAN: {
        const double c = 2.772588722239781 / (S.irc_fwhm * S.irc_fwhm);
        return sqrt(c / 3.14159265358979323846) * exp(-c * x * x);
    }
    case HEART_IRC_LORENTZIAN:
        return S.irc_fwhm / (2.0 * 3.14159265358979323846) / (0.25 * S.irc_fwhm * S.irc_fwhm + x * x);
    default:
        return fabs(x) <= 0.5 * S.irc_fwhm ? 1.0 / S.irc_fwhm : 0.0;
    }
}

// W(q) / W(0) of the mosaic distribution, q = 1 - cos(theta) (the closed forms
// set up by the host: theta shapes, vMF, WL, SWL, uniform)
__device__ __forceinline__ double mdf_ratio64(const SpecParams &S, double q) {
    switch (S.mdf) {
    case HEART_MDF_VMF: return exp(-S.w_c * q);
    case HEART_MDF_WRAPPED_LORENTZIAN: return S.w_a2 / (S.w_a2 + 2.0 * q);
    case HEART_MDF_SPHERICAL_WRAPPED_LORENTZIAN: {
        const double r = S.w_b / (S.w_b + q);
        return r * r;
    }
    case HEART_MDF_UNIFORM: return q <= S.w_qmax ? 1.0 : 0.0;
    default: {
        const double th = 2.0 * asin(sqrt(0.5 * fmin(fmax(q, 0.0), 2.0)));
        return S.w_wl * (S.w_a2 / (S.w_a2 + th * th)) + S.w_wg * exp(-S.w_c * th * th);
    }
    }
}

// unit vectors perpendicular to k: e1 along the part of N perpendicular to k
// (t1's part when k is along N), e2 = k x e1
__device__ __forceinline__ void cone_axes64(const double k[3], const double N[3], const double t1[3], double e1[3],
                                            double e2[3]) {
    const double kN = dot3d(k, N);
    for (int i = 0; i < 3; ++i) e1[i] = N[i] - kN * k[i];
    double n2 = dot3d(e1, e1);
    if (!(n2 > 1e-300)) {
        const double kt = dot3d(k, t1);
        for (int i = 0; i < 3; ++i) e1[i] = t1[i] - kt * k[i];
        n2 = dot3d(e1, e1);
    }
    const double inv = 1.0 / sqrt(n2);
    for (int i = 0; i < 3; ++i) e1[i] *= inv;
    e2[0] = k[1] * e1[2] - k[2] * e1[1];
    e2[1] = k[2] * e1[0] - k[0] * e1[2];
    e2[2] = k[0] * e1[1] - k[1] * e1[0];
}

// entry point on the front face; true on a hit
__device__ __forceinline__ bool entry64(const SpecParams &S, const double o[3], const double k[3], double p[3]) {
    const double rel[3] = {o[0] - S.c[0], o[1] - S.c[1], o[2] - S.c[2]};
    if (S.geometry == HEART_FLAT) {
        const double h0 = dot3d(rel, S.N), kN = dot3d(k, S.N);
        if (!(kN < 0) || !(h0 > 0)) return false;
        const double t = h0 / (-kN);
        for (int i = 0; i < 3; ++i) p[i] = o[i] + t * k[i];
        const double r2[3] = {p[0] - S.c[0], p[1] - S.c[1], p[2] - S.c[2]};
        return fabs(dot3d(r2, S.ed)) <= S.half_d && fabs(dot3d(r2, S.en)) <= S.half_n;
    }
    const double X = dot3d(rel, S.cc), Y = dot3d(rel, S.ww);
    const double kX = dot3d(k, S.cc), kY = dot3d(k, S.ww);
    const double c = X * X + Y * Y - S.radius * S.radius;
    if (!(c < 0)) return false;
    const double a = kX * kX + kY * kY;
    if (!(a > 0)) return false;
    const double b = X * kX + Y * kY;
    const double sq = sqrt(b * b - a * c);
    const double t = (b > 0) ? -c / (b + sq) : (-b + sq) / a;
    for (int i = 0; i < 3; ++i) p[i] = o[i] + t * k[i];
    const double r2[3] = {p[0] - S.c[0], p[1] - S.c[1], p[2] - S.c[2]};
    const double z = dot3d(r2, S.ax), Xp = dot3d(r2, S.cc), Yp = dot3d(r2, S.ww);
    return fabs(z - S.zc) <= S.half_d && fabs(Yp) * S.cphi <= Xp * S.sphi;
}

// distance from p (inside) along k to the first boundary crossing, and the face
__device__ __forceinline__ double exit_distance64(const SpecParams &S, const double p[3], const double k[3],
                                                  int *face) {
    const double rel[3] = {p[0] - S.c[0], p[1] - S.c[1], p[2] - S.c[2]};
    double best = 1e300;
    int f = HEART_EXIT_SIDE;
    auto cand = [&](double v, int fc) {
        v = v < 0 ? 0 : v;
        if (v < best) { best = v; f = fc; }
    };
    if (S.geometry == HEART_FLAT) {
        const double h = dot3d(rel, S.N), a = dot3d(rel, S.ed), b = dot3d(rel, S.en);
        const double kh = dot3d(k, S.N), ka = dot3d(k, S.ed), kb = dot3d(k, S.en);
        if (kh > 0) cand((0.0 - h) / kh, HEART_EXIT_FRONT);
        if (kh < 0) cand((-S.thickness - h) / kh, HEART_EXIT_BACK);
        if (ka > 0) cand((S.half_d - a) / ka, HEART_EXIT_SIDE);
        if (ka < 0) cand((-S.half_d - a) / ka, HEART_EXIT_SIDE);
        if (kb > 0) cand((S.half_n - b) / kb, HEART_EXIT_SIDE);
        if (kb < 0) cand((-S.half_n - b) / kb, HEART_EXIT_SIDE);
    } else {
        const double z = dot3d(rel, S.ax), X = dot3d(rel, S.cc), Y = dot3d(rel, S.ww);
        const double kz = dot3d(k, S.ax), kX = dot3d(k, S.cc), kY = dot3d(k, S.ww);
        const double R = S.radius, Ro = S.radius + S.thickness;
        const double a = kX * kX + kY * kY, b = X * kX + Y * kY;
        if (a > 0) {
            const double ci = X * X + Y * Y - R * R;
            if (b < 0) {
                const double disc = b * b - a * ci;
                if (disc >= 0) cand(ci / (-b + sqrt(disc)), HEART_EXIT_FRONT);
            }
            const double co = X * X + Y * Y - Ro * Ro;
            double disc = b * b - a * co;
            disc = disc < 0 ? 0 : disc;
            const double sq = sqrt(disc);
            cand((b > 0) ? -co / (b + sq) : (-b + sq) / a, HEART_EXIT_BACK);
        }
        if (kz > 0) cand((S.zc + S.half_d - z) / kz, HEART_EXIT_SIDE);
        if (kz < 0) cand((S.zc - S.half_d - z) / kz, HEART_EXIT_SIDE);
        const double gp = -X * S.sphi + Y * S.cphi, rp = -kX * S.sphi + kY * S.cphi;
        if (rp > 0) cand(-gp / rp, HEART_EXIT_SIDE);
        const double gm = -X * S.sphi - Y * S.cphi, rm = -kX * S.sphi - kY * S.cphi;
        if (rm > 0) cand(-gm / rm, HEART_EXIT_SIDE);
    }
    *face = f;
    return best;
}

__device__ __forceinline__ void local_frame64(const SpecParams &S, const double p[3], double N[3], double t1[3],
                                              double t2[3]) {
    if (S.geometry == HEART_FLAT) {
        for (int i = 0; i < 3; ++i) { N[i] = S.N[i]; t1[i] = S.ed[i]; t2[i] = S.en[i]; }
        return;
    }
    const double rel[3] = {p[0] - S.c[0], p[1] - S.c[1], p[2] - S.c[2]};
    const double X = dot3d(rel, S.cc), Y = dot3d(rel, S.ww);
    const double inv = 1.0 / sqrt(X * X + Y * Y);
    for (int i = 0; i < 3; ++i) { N[i] = -(X * S.cc[i] + Y * S.ww[i]) * inv; t1[i] = S.ax[i]; }
    t2[0] = N[1] * t1[2] - N[2] * t1[1];
    t2[1] = N[2] * t1[0] - N[0] * t1[2];
    t2[2] = N[0] * t1[1] - N[1] * t1[0];
}

__device__ __forceinline__ void detector64(const SpecParams &S, const double x[3], const double k[3], RayOut64 &r) {
    const double den = dot3d(k, S.nd);
    if (den == 0) return;
    const double rel[3] = {S.D0[0] - x[0], S.D0[1] - x[1], S.D0[2] - x[2]};
    const double t = dot3d(rel, S.nd) / den;
    if (!(t > 0)) return;
    const double P[3] = {x[0] + t * k[0] - S.D0[0], x[1] + t * k[1] - S.D0[1], x[2] + t * k[2] - S.D0[2]};
    r.u = dot3d(P, S.eu);
    r.v = dot3d(P, S.ev);
    const double fx = r.u / S.pix + 0.5 * S.nx, fy = r.v / S.pix + 0.5 * S.ny;
    if (fx >= 0 && fx < S.nx && fy >= 0 && fy < S.ny) {
        r.ix = (int)floor(fx);
        r.iy = (int)floor(fy);
        r.det_hit = 1;
    }
}

// ---------------------------------------------------------------------------
// thinned candidates (FP64): bounds of one straight segment.  The scatter
// candidates of the majorant walk split by their marks (v, n) into (a) v < v*,
// tested as usual; (b) v >= v*, tilt q in [q_min, 2 - q_min], azimuth in the
// arcs where |Delta| < X*, tested as usual; (c) the rest, which cannot reflect
// and are never drawn.  On the segment the grazing angle stays in
// [a_lo, a_hi]; a tilt theta < d - X* (d: distance of alpha_B + Delta_M from
// that range) keeps |Delta| >= X*.  Segments with d <= X* keep the plain stream.
// ---------------------------------------------------------------------------
// per-ray constants of the reflection orders (Eq. BraggLaw on d / m_h, Q_h,
// the rocking curve's width scale, and Q_h R_max / w_h, the order's share of
// the majorant), and the energy-dependent peak shift
struct Orders64 {
    int n;
    double shift;
    double alpha[HEART_MAX_ORDERS], Q[HEART_MAX_ORDERS], w[HEART_MAX_ORDERS], qr[HEART_MAX_ORDERS];
};

// the energy-dependent rocking curve at E: width scale and added shift, linear
// between the knots and constant beyond them
__host__ __device__ __forceinline__ void irc_energy64(const SpecParams &S, double E, double &ws, double &sh) {
    ws = 1.0;
    sh = 0.0;
    const int n = S.n_irc_e;
    if (n <= 0) return;
    if (n == 1 || E <= S.irc_e[0]) { ws = S.irc_ws[0]; sh = S.irc_sh[0]; return; }
    if (E >= S.irc_e[n - 1]) { ws = S.irc_ws[n - 1]; sh = S.irc_sh[n - 1]; return; }
    int i = 0;
    while (!(E < S.irc_e[i + 1])) ++i;
    const double f = (E - S.irc_e[i]) / (S.irc_e[i + 1] - S.irc_e[i]);
    ws = S.irc_ws[i] + f * (S.irc_ws[i + 1] - S.irc_ws[i]);
    sh = S.irc_sh[i] + f * (S.irc_sh[i + 1] - S.irc_sh[i]);
}

struct Bound64 {
    double ra, vstar, qmin, pbar, S1, S2, lam;
    unsigned long long w0, wspan;
    unsigned long long w1, w2;     // band B of process (b): table words [w1, w2) (w1 = w2 = w0: none)
    double pbarB, sA;              // band B's arc-measure bound; band A's share of process (b)
    // no rocking curve, thinned: W / W(0) bounds of the two cones, the facing cone's window
    // |psi| < psis, and the cumulative shares of the window and of the whole facing cone
    double wn, wf, psis, pin, pio;
};

struct Seg64 {
    double mu, pa;
    double cum[HEART_MAX_ORDERS];
    Bound64 o[HEART_MAX_ORDERS];
};

// the tilt-grid point just below q_min (-1 below the grid)
__device__ __forceinline__ int tilt_index64(double qmin) {
    if (!(qmin >= 3.552713678800501e-15)) return -1;                   // 2^-48
    const int j = (int)floor(8.0 * log2(qmin)) + 384;
    return j > kQGrid - 1 ? kQGrid - 1 : j;
}

// Band B's arc-measure bound (units of pi) for tilts q in [q1, q2] on a segment
// with |k.N| in [lo, hi]: with b = c_a sin(theta), the window's interval of
// cos(xi') on the ray's side, (S - a (1 - q)) / b, stays within |y| <= M =
// D / (c_a,min sin theta1) + hi tan(theta2 / 2) / c_a,min (D = max |S - a|), where
// an interval's arcsine measure is at most its width over sqrt(1 - M^2); the other
// one lies beyond m = (S1 + lo (1 - q2)) / sin theta2 (measure <= acos m,
// 0 if m >= 1); w = (S2 - S1) / (c_a,min sin theta1)
__device__ __forceinline__ double band_b_bound64(double lo, double hi, double S1, double S2, double q1, double q2) {
    const double h = fmin(hi, 1.0);
    const double camin = sqrt(fmax(0.0, 1.0 - h * h));
    const double s1 = sqrt(q1 * (2.0 - q1)), s2 = sqrt(q2 * (2.0 - q2)), t2 = sqrt(q2 / (2.0 - q2));
    if (!(camin > 0.0) || !(s1 > 0.0)) return 1.0;
    const double D = fmax(fabs(S1 - hi), fabs(S2 - lo));
    const double M = D / (camin * s1) + hi * t2 / camin;
    const double w = (S2 - S1) / (camin * s1);
    if (!(M < 1.0)) return 1.0;
    const double same = w / sqrt(1.0 - M * M);
    const double m = (S1 + lo * (1.0 - q2)) / s2;
    const double mirror = m >= 1.0 ? 0.0 : acos(fmax(-1.0, m));
    return (same + mirror) / 3.14159265358979323846;
}

// the thinning bound of order h on a segment with |k.N| in [lo, hi]
__device__ __forceinline__ void bound_order64(const SpecParams &S, const Orders64 &O, int h, double lo, double hi,
                                              Bound64 &b) {
    b.ra = 1.0; b.vstar = 1.0; b.qmin = 0.0; b.pbar = 1.0; b.S1 = 0.0; b.S2 = 0.0;
    b.w0 = 0ull; b.wspan = 1ull << 32;
    b.w1 = 0ull; b.w2 = 0ull; b.pbarB = 1.0; b.sA = 1.0;
    b.lam = O.qr[h];
    b.wn = 1.0; b.wf = 1.0; b.psis = 3.14159265358979323846; b.pin = 0.5; b.pio = 0.5;
    if (S.sampler == HEART_SAMPLER_THINNED && S.irc == HEART_IRC_NONE && O.qr[h] > 0) {
        // no rocking curve: the facing cone's crystallites are tilted by at least d
        // (distance of sin a~0 from the segment's |k.N| range), the other cone's by at
        // least a~0; W there, relative to W(0), bounds each cone on the segment
        const double a0 = O.alpha[h] + O.shift, s0 = sin(a0);
        const double d = s0 < lo ? lo - s0 : (s0 > hi ? s0 - hi : 0.0);
        const double hn = sin(0.5 * d), hf = sin(0.5 * a0);
        const double q0 = 2.0 * hn * hn;
        b.wn = mdf_ratio64(S, q0);
        b.wf = mdf_ratio64(S, 2.0 * hf * hf);
        // on the facing cone q(psi) >= q0 + cos(a~0) cos(g_max) (1 - cos psi): W <= v* W(0)
        // outside |psi| < psis
        const double sh = fmin(hi, 1.0), cmin = cos(a0) * sqrt(1.0 - sh * sh);
        if (q0 < S.none_qv && cmin > 0) {
            const double xq = (S.none_qv - q0) / cmin;
            if (xq < 2.0) b.psis = 2.0 * asin(sqrt(0.5 * xq));
        }
        const double pi = 3.14159265358979323846;
        const double fin = b.wn * (b.psis / pi), fout = b.psis < pi ? S.vstar * (1.0 - b.psis / pi) : 0.0;
        const double tot = fin + fout + b.wf;
        b.lam = 0.5 * O.qr[h] * tot;
        b.pin = tot > 0 ? fin / tot : 1.0;
        b.pio = tot > 0 ? (fin + fout) / tot : 1.0;
        return;
    }
    if (S.sampler != HEART_SAMPLER_THINNED || S.irc == HEART_IRC_NONE || !(O.qr[h] > 0)) return;
    // distance between sines: never more than between the angles
    const double aBs = O.alpha[h] + O.shift;
    const double xstar = S.xstar * O.w[h];                 // a curve w times as wide: X* scales by w
    const double sBs = sin(aBs);
    const double d = sBs < lo ? lo - sBs : (sBs > hi ? sBs - hi : 0.0);
    double tmin = d - xstar;
    if (!(tmin > 0)) return;
    const double half_pi = 1.5707963267948966;
    if (tmin > half_pi) tmin = half_pi;
    const double sh = sin(0.5 * tmin);
    b.qmin = 2.0 * sh * sh;
    const int j0 = tilt_index64(b.qmin);
    b.w0 = j0 < 0 ? 0ull : (unsigned long long)S.qgrid[j0];
    b.wspan = (1ull << 32) - b.w0;
    b.S1 = sin(fmax(0.0, aBs - xstar));
    b.S2 = sin(fmin(half_pi, aBs + xstar));
    const double hc = fmin(hi, 1.0);
    const double bmin = sqrt(fmax(0.0, 1.0 - hc * hc)) * sin(tmin);
    // two windows of width w in cos(xi'), each of arc measure <= acos(1 - w) / pi
    const double w = (b.S2 - b.S1) / bmin;
    b.pbar = (w >= 2.0 || !(bmin > 0)) ? 1.0 : fmin(1.0, 2.0 * acos(1.0 - w) / 3.14159265358979323846);
    b.w1 = b.w2 = b.w0;
    b.pbarB = b.pbar;
    if (O.n == 1 && j0 >= 0 && j0 + kBandDJ < kBandJ2) {
        const unsigned long long w1 = S.qgrid[j0 + kBandDJ], w2 = S.qgrid[kBandJ2];
        if (w1 < w2) {
            // the band's tilts: from the table knot that starts w1's interval to q_J
            const double pB = band_b_bound64(lo, hi, b.S1, b.S2, S.mdf64[w1 >> 20], exp2(kBandJ2 / 8.0 - 48.0));
            if (pB < b.pbar) {
                b.w1 = w1;
                b.w2 = w2;
                b.pbarB = pB;
            }
        }
    }
    const double QR = O.qr[h];
    const double PA = (double)((b.w1 - b.w0) + ((1ull << 32) - b.w2)) / 4294967296.0;
    const double PB = (double)(b.w2 - b.w1) / 4294967296.0;
    const double lA = PA * b.pbar, lB = PB * b.pbarB;
    b.sA = lA + lB > 0.0 ? lA / (lA + lB) : 1.0;
    const double la = QR * S.vstar, lb = QR * (1.0 - S.vstar) * (lA + lB);
    b.vstar = S.vstar;
    b.lam = la + lb;
    b.ra = la / (la + lb);
}

__device__ __forceinline__ void bound_segment64(const SpecParams &S, const Orders64 &O, double mu0, bool any_bragg,
                                                const double x[3], const double k[3], Seg64 &b) {
    double lo = 0.0, hi = 1.0;
    if (S.sampler == HEART_SAMPLER_THINNED && any_bragg) {
        int face;
        const double se = exit_distance64(S, x, k, &face);
        double xe[3], N0[3], N1[3], t1[3], t2[3];
        for (int i = 0; i < 3; ++i) xe[i] = x[i] + se * k[i];
        local_frame64(S, x, N0, t1, t2);
        local_frame64(S, xe, N1, t1, t2);
        const double k0 = dot3d(k, N0), k1 = dot3d(k, N1);
        lo = fmin(fabs(k0), fabs(k1));
        hi = fmax(fabs(k0), fabs(k1));
        if ((k0 < 0) != (k1 < 0)) lo = 0.0;                // k.N is monotone along a line
    }
    double lam = 0.0;
    for (int h = 0; h < O.n; ++h) {
        bound_order64(S, O, h, lo, hi, b.o[h]);
        lam += b.o[h].lam;
    }
    double run = 0.0;
    for (int h = 0; h < O.n; ++h) {
        run += b.o[h].lam;
        b.cum[h] = lam > 0 ? run / lam : 1.0;
    }
    b.cum[O.n - 1] = 1.0;
    b.mu = mu0 + lam;
    b.pa = mu0 / b.mu;
}

// arc measure (in units of pi) of xi' in [0, pi] with |a + b cos xi'| in (S1, S2), and the arcs
__device__ __forceinline__ double azimuth_arcs64(double a, double b, double S1, double S2, double arc[4]) {
    const double iv[2][2] = {{(S1 - a) / b, (S2 - a) / b}, {(-S2 - a) / b, (-S1 - a) / b}};
    double tot = 0.0;
    for (int j = 0; j < 2; ++j) {
        const double l = fmax(-1.0, iv[j][0]), h = fmin(1.0, iv[j][1]);
        arc[2 * j] = 0.0;
        arc[2 * j + 1] = 0.0;
        if (l < h) {
            arc[2 * j] = acos(h);
            arc[2 * j + 1] = acos(l) - acos(h);
            tot += arc[2 * j + 1];
        }
    }
    return tot / 3.14159265358979323846;
}

// one ray, source (or user arrays) to detector
__device__ inline void trace_ray64(const SpecParams &S, const SourceParams &P, uint32_t k0, uint32_t k1,
                                   uint64_t ray, uint64_t idx, const double *tab, RayOut64 &r) {
    constexpr double kTwoPi = 6.283185307179586476925;
    const uint32_t rl = (uint32_t)ray, rh = (uint32_t)(ray >> 32);
    r.outcome = HEART_MISS; r.nrefl = 0; r.ncoll = 0; r.ix = -1; r.iy = -1; r.det_hit = 0; r.no_bragg = 0;
    r.u = __longlong_as_double(0x7ff8000000000000LL);
    r.v = r.u;
    double E, k[3], o[3], pv[3] = {0.0, 0.0, 0.0};
    int pol = 0;
    if (P.user) {
        E = P.ray[6][idx];
        for (int i = 0; i < 3; ++i) { o[i] = P.ray[i][idx]; k[i] = P.ray[3 + i][idx]; }
        const double kk = sqrt(dot3d(k, k));
        if (kk > 0) for (int i = 0; i < 3; ++i) k[i] /= kk;
        else E = __longlong_as_double(0x7ff8000000000000LL);     // a zero direction cannot enter
        if (P.pol_on) {
            const double p0[3] = {P.ray[7][idx], P.ray[8][idx], P.ray[9][idx]};
            pol = project_pol64(p0, k, pv);
        }
    } else {
    uint32_t a[4], b[4];
    philox4x32_10(rl, rh, 0u, 0u, k0, k1, a);
    philox4x32_10(rl, rh, 1u, 0u, k0, k1, b);

    // a: call 0, the spot and the direction (all the entry test needs); b: call 1,
    // the energy's words (Sec. 2.1 draws them as independent uniforms)
    // energy (Sec. 2.1): component by cumulative weight, then its parameter
    const double uc = u01_64(b[0]);
    int c = P.n_comp - 1;
    for (int i = 0; i < P.n_comp; ++i)
        if (uc < P.cumw[i]) { c = i; break; }
    const double up = u01_64(b[1]);
    switch (P.kind[c]) {
    case HEART_SRC_MONO: E = P.e0[c]; break;
    case HEART_SRC_GAUSS:
        E = P.e0[c] + P.width[c] * (sqrt(-2.0 * log(u01_64(b[2]))) * cos(kTwoPi * u01_64(b[3])));
        break;
    case HEART_SRC_LORENTZ: {
        const double uu = P.lorentz_F0[c] + up * (1.0 - P.lorentz_F0[c]);
        E = P.e0[c] + 0.5 * P.width[c] * tan(3.14159265358979323846 * (uu - 0.5));
        break;
    }
    case HEART_SRC_INV_E: E = P.lo[c] * pow(P.hi[c] / P.lo[c], up); break;
    case HEART_SRC_TABLE: {
        // inverse of the piecewise-linear CDF: the interval with C_i <= up < C_i+1
        int lo = 0, hi = P.n_tab - 1;
        while (hi - lo > 1) {
            const int m = (lo + hi) >> 1;
            if (up < P.tab_cdf[m]) hi = m; else lo = m;
        }
        const double *C = P.tab_cdf, *x = P.tab_keV;
        E = x[lo] + (up - C[lo]) / (C[lo + 1] - C[lo]) * (x[lo + 1] - x[lo]);
        break;
    }
    default: E = P.lo[c] + (P.hi[c] - P.lo[c]) * up; break;
    }
    // direction uniform in solid angle inside the cone
    const double w = u01_64(a[2]) * P.one_minus_cos_max;
    const double cphi = 1.0 - w, sphi = sqrt(w * (2.0 - w));
    const double beta = kTwoPi * u01_64(a[3]);
    const double cb = cos(beta), sb = sin(beta);
    for (int i = 0; i < 3; ++i) k[i] = cphi * P.ax[i] + sphi * (cb * P.b1[i] + sb * P.b2[i]);
    // Gaussian spot
    const double rr = sqrt(-2.0 * log(u01_64(a[0])));
    const double ang = kTwoPi * u01_64(a[1]);
    const double z1 = rr * cos(ang), z2 = rr * sin(ang);
    for (int i = 0; i < 3; ++i) o[i] = P.origin[i] + P.sig1 * z1 * P.b1[i] + P.sig2 * z2 * P.b2[i];
    if (P.pol_on) pol = project_pol64(P.pol, k, pv);
    }
    r.E = E;

    double x[3];
    const bool hit = (E > 0 && isfinite(E)) && entry64(S, o, k, x);
    if (!hit) {
        for (int i = 0; i < 3; ++i) { r.pos[i] = o[i]; r.dir[i] = k[i]; r.pol[i] = pol ? pv[i] : 0.0; }
        return;
    }
    // per-ray constants of each reflection order: Bragg angle (Eq. BraggLaw on
    // d / m_h), Q_h, the rocking curve's width scale at E and its share of the
    // majorant Q_h R_max / w_h; mu0 and the peak shift at E
    const double lam_A = 12.398419843320026 / E;
    const double mu0 = 1.0 / (S.labs * pow(E / S.labs_ref, S.labs_pow));
    Orders64 O;
    O.n = S.n_orders;
    double ws, shE;
    irc_energy64(S, E, ws, shE);
    O.shift = S.irc_shift + shE;
    bool any_bragg = false;
    for (int h = 0; h < O.n; ++h) {
        const double sb = S.ord_m[h] * lam_A / (2.0 * S.d_A);
        O.w[h] = S.ord_w[h] * ws;
        O.alpha[h] = 0.0;
        O.Q[h] = 0.0;
        O.qr[h] = 0.0;
        if (!(sb < 1.0)) continue;
        any_bragg = true;
        O.alpha[h] = asin(sb);
        const double lam = lam_A * 1e-7;
        const double Kh = S.K * S.ord_k[h];
        O.Q[h] = Kh * Kh * lam * lam * lam / (2.0 * sb * sqrt(1.0 - sb * sb));
        O.qr[h] = O.Q[h] * (S.irc_max / O.w[h]);        // a curve w times as wide peaks 1/w as high
        if (S.irc == HEART_IRC_NONE) {
            // no rocking curve: Q cos a~0 x 2 cones x 2 pi f(0), a~0 = aB + Delta_M
            const double a0 = O.alpha[h] + O.shift;
            O.qr[h] = (a0 > 0.0 && a0 < 1.5707963267948966) ? O.Q[h] * cos(a0) * S.none_fac : 0.0;
        }
    }
    if (!any_bragg) r.no_bragg = 1;

    // null-collision walk (Sec. 2.2.4), candidates thinned per straight segment
    int outcome = HEART_STUCK, nrefl = 0;
    long long ncoll = 0;
    uint32_t call = 2;
    Seg64 sb;
    bound_segment64(S, O, mu0, any_bragg, x, k, sb);
    for (;;) {
        if (ncoll >= S.max_coll) { outcome = HEART_STUCK; break; }
        uint32_t wd[4];
        philox4x32_10(rl, rh, call++, 0u, k0, k1, wd);
        const double l = -log(u01_64(wd[0])) / sb.mu;
        int face;
        const double se = exit_distance64(S, x, k, &face);
        if (l > se) {
            for (int i = 0; i < 3; ++i) x[i] += se * k[i];
            outcome = face;
            break;
        }
        for (int i = 0; i < 3; ++i) x[i] += l * k[i];
        ++ncoll;
        const double u1 = u01_64(wd[1]);
        if (u1 < sb.pa) { outcome = HEART_ABSORBED; break; }
        double v = (u1 - sb.pa) / (1.0 - sb.pa);
        // the reflection order by its share of the candidate rate (sum over H);
        // the conditional uniform stays the acceptance uniform
        int h = 0;
        if (O.n > 1) {
            while (h < O.n - 1 && !(v < sb.cum[h])) ++h;
            const double c0 = h > 0 ? sb.cum[h - 1] : 0.0;
            v = (v - c0) / (sb.cum[h] - c0);
        }
        double ks[3], P;                                      // reflected direction, acceptance probability
        double N[3], t1[3], t2[3];
        local_frame64(S, x, N, t1, t2);
        if (S.irc == HEART_IRC_NONE) {
            // no rocking curve: the crystallite normal on the cone k.n = sg sin a~0
            // (sg by the top bit of u2) at azimuth psi = 2 pi u3 about k
            const double a0 = O.alpha[h] + O.shift, s0 = sin(a0), c0 = cos(a0);
            double sg, wb = 1.0;                                // the cone, and its bound of W / W(0)
            double x2 = 2.0 * u01_64(wd[3]);                    // psi / pi
            if (S.sampler == HEART_SAMPLER_THINNED) {
                // the facing cone (k.n of the sign of k.N): its window |psi| < psis or the
                // rest; or the other cone; by their shares of the bound
                const Bound64 &ob = sb.o[h];
                const double side = dot3d(k, N) < 0 ? -1.0 : 1.0, u2 = u01_64(wd[2]), u3 = u01_64(wd[3]);
                const double pi = 3.14159265358979323846;
                if (u2 < ob.pin) {
                    sg = side; wb = ob.wn; x2 = ob.psis * (2.0 * u3 - 1.0) / pi;
                } else if (u2 < ob.pio) {
                    sg = side; wb = S.vstar; x2 = (ob.psis + 2.0 * (pi - ob.psis) * u3) / pi;
                } else {
                    sg = -side; wb = ob.wf;
                }
            } else {
                sg = (wd[2] & 0x80000000u) ? 1.0 : -1.0;
            }
            double sp, cp, e1[3], e2[3], n[3];
            sincospi(x2, &sp, &cp);
            cone_axes64(k, N, t1, e1, e2);
            for (int i = 0; i < 3; ++i) n[i] = sg * s0 * k[i] + c0 * (cp * e1[i] + sp * e2[i]);
            const double q = 1.0 - dot3d(n, N);                 // the crystallite's tilt, 1 - cos(theta)
            for (int i = 0; i < 3; ++i) ks[i] = k[i] - 2.0 * (sg * s0) * n[i];
            double G;
            if (pol) {
                const double pk = dot3d(pv, ks);
                G = 1.0 - pk * pk;
            } else {
                const double c2 = cos(2.0 * a0);
                G = 0.5 * (1.0 + c2 * c2);
            }
            P = mdf_ratio64(S, q) / wb * G;
        } else {
        const Bound64 &ob = sb.o[h];
        double q, sx, cx;
        if (v < ob.ra) {                                      // process (a), or the plain stream
            v = ob.ra < 1.0 ? (v / ob.ra) * ob.vstar : v;
            q = mdf_q64(tab, wd[2]);
            sincospi(2.0 * u01_64(wd[3]), &sx, &cx);
        } else {                                              // process (b)
            double vb = (v - ob.ra) / (1.0 - ob.ra), pb;
            unsigned long long wq;
            if (vb < ob.sA) {                                 // band A: words [w0, w1) and [w2, 2^32)
                if (ob.sA < 1.0) vb /= ob.sA;
                const unsigned long long span = (ob.w1 - ob.w0) + ((1ull << 32) - ob.w2);
                wq = ob.w0 + (((unsigned long long)wd[2] * span) >> 32);
                if (wq >= ob.w1) wq += ob.w2 - ob.w1;
                pb = ob.pbar;
            } else {                                          // band B: words [w1, w2)
                vb = (vb - ob.sA) / (1.0 - ob.sA);
                wq = ob.w1 + (((unsigned long long)wd[2] * (ob.w2 - ob.w1)) >> 32);
                pb = ob.pbarB;
            }
            v = ob.vstar + (1.0 - ob.vstar) * vb;
            q = mdf_q64(tab, (uint32_t)wq);
            if (q < ob.qmin || q > 2.0 - ob.qmin) continue;  // cannot reflect
            const double kN = dot3d(k, N), sa_ = fabs(kN), ca_ = sqrt(fmax(0.0, 1.0 - kN * kN));
            const double a = (kN < 0 ? -sa_ : sa_) * (1.0 - q), b = ca_ * sqrt(q * (2.0 - q));
            double arc[4];
            const double Pxi = azimuth_arcs64(a, b, ob.S1, ob.S2, arc);
            const double t3 = u01_64(wd[3]);
            if (!(t3 * pb < Pxi)) continue;                   // outside the arcs: cannot reflect
            const double L = arc[1] + arc[3];
            double pos = (t3 * pb / Pxi) * 2.0 * L, sgn = 1.0;
            if (pos >= L) { pos -= L; sgn = -1.0; }
            const double xp = pos < arc[1] ? arc[0] + pos : arc[2] + (pos - arc[1]);
            sincos(atan2(dot3d(k, t2), dot3d(k, t1)) + sgn * xp, &sx, &cx);
        }
        const double ct = 1.0 - q, st = sqrt(q * (2.0 - q));
        double n[3];
        for (int i = 0; i < 3; ++i) n[i] = ct * N[i] + st * (cx * t1[i] + sx * t2[i]);
        const double kn = dot3d(k, n);
        double sa = fabs(kn);
        sa = sa > 1.0 ? 1.0 : sa;
        const double delta = asin(sa) - O.alpha[h] - O.shift;
        for (int i = 0; i < 3; ++i) ks[i] = k[i] - 2.0 * kn * n[i];   // reflected direction
        double G;
        if (pol) {
            const double pk = dot3d(pv, ks);
            G = 1.0 - pk * pk;                                // Eq. (G_pol): 1 - (p . k_s)^2
        } else {
            const double c2 = 1.0 - 2.0 * sa * sa;            // cos(2 a~)
            G = 0.5 * (1.0 + c2 * c2);                        // Eq. (G_unpol)
        }
        // order h's curve is the described one w_h times as wide: R_h / R_h,max = R(x / w_h) / R_max
        P = irc64(S, delta / O.w[h]) * G / S.irc_max;
        }
        if (v < P) {
            ++nrefl;
            if (nrefl > S.max_refl) { outcome = HEART_CAPPED; break; }
            const double inv = 1.0 / sqrt(dot3d(ks, ks));
            for (int i = 0; i < 3; ++i) k[i] = ks[i] * inv;
            if (pol) {                                        // p_s = (p - (p.k_s) k_s) / |...|
                const double pk = dot3d(pv, k);
                const double d = 1.0 / sqrt(1.0 - pk * pk);
                for (int i = 0; i < 3; ++i) pv[i] = (pv[i] - pk * k[i]) * d;
                const double pn = 1.0 / sqrt(dot3d(pv, pv));
                for (int i = 0; i < 3; ++i) pv[i] *= pn;
            }
            bound_segment64(S, O, mu0, any_bragg, x, k, sb);   // a new straight segment
        }
    }
    r.outcome = outcome;
    r.nrefl = nrefl;
    r.ncoll = ncoll;
    for (int i = 0; i < 3; ++i) { r.pos[i] = x[i]; r.dir[i] = k[i]; r.pol[i] = pol ? pv[i] : 0.0; }
    if (outcome == HEART_EXIT_FRONT || outcome == HEART_EXIT_BACK || outcome == HEART_EXIT_SIDE)
        detector64(S, x, k, r);
}

}  // namespace heart
