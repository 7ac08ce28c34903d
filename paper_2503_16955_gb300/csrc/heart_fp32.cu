// heart_fp32.cu -- the FP32 persistent ray-transport kernel.
//
// Precision plan (Sec. 2.2.3-2.2.4 of the paper fix what is computed; this
// file fixes how):
//  * per ray and per straight segment (entry, after each reflection) the
//    direction k, the segment start x0 and sin(aB + Delta_M) are held in FP64,
//    and the Bragg anchor A = |k.N(x0)| - sin(aB + Delta_M) is formed in FP64;
//  * per tentative collision everything is FP32, and only *small* quantities
//    are formed: the candidate offset D = k.n - k.N (size ~ theta), the
//    along-segment change of k.N on a cylinder, and the rocking-curve argument
//    Delta = asin(s) - asin(sB) = asin((s - sB)(s + sB) / (s cB + sB cs)) with
//    s - sB = A + sign * (D + dkappa); no large number is ever subtracted in FP32;
//  * the path length along a segment is a Kahan-compensated FP32 sum.
// Decisions that compare a uniform with a per-ray threshold (absorption,
// spectral component) compare the raw 32-bit Philox word with an integer
// threshold, so they agree with the FP64 path exactly.
//
// Work distribution: a persistent grid; each warp owns a shared-memory buffer
// of spawned rays (source sampled, crystal entry found, misses already tallied).
// All 32 lanes spawn together (full SIMT efficiency) when the buffer runs low;
// lanes whose ray ended pop a new ray from the buffer once at least
// `refill` lanes are idle, so the expensive spawn never runs divergently.
#include <cuda_runtime.h>

#include <cstring>

#include "heart_fp64.cuh"
#include "heart_lib.h"

namespace heart {

constexpr int kWarpsPerBlock = 4;
constexpr int kBlockThreads = kWarpsPerBlock * 32;
constexpr int kBuf = 64;                 // spawned rays buffered per warp

// Per-launch parameters in the crystal-local frame.
// flat: axes (e_d, e_n, N), origin at the front-face centre; crystal
//       |p0| <= half_d, |p1| <= half_n, -t <= p2 <= 0.
// cylinder: axes (axis, c, axis x c), origin on the axis; crystal
//       |p0 - zc| <= half_d, R <= hypot(p1, p2) <= R + t, |p2| cphi <= p1 sphi.
struct Launch32 {
    // source, local frame
    double o[3], ax[3], b1[3], b2[3];
    float omc, sig1, sig2;
    int32_t n_comp;
    uint32_t comp_thr[kMaxComp];          // component i if word < comp_thr[i]
    int32_t kind[kMaxComp];
    double e0[kMaxComp];
    float width[kMaxComp], lo[kMaxComp], hi[kMaxComp], lF0[kMaxComp];
    // crystal
    float half_d, half_n, thick, R, zc, sphi, cphi;
    double R64, zc64, cos_shift;
    float sin_shift;
    // rocking curve (argument x = Delta - Delta_M)
    float irc_fwhm, irc_eta, irc_delta, irc_inv_norm, irc_g, inv_irc_max, irc_c, irc_gnorm;
    // physics
    double sB_scale;                      // hc / (2 d)   [keV]
    float labs, labs_ref, labs_pow, K2, irc_max;
    int32_t max_refl;
    int64_t max_coll;
    // detector, local frame
    double D0[3];
    float eu[3], ev[3], nd[3], inv_pix, hnx, hny;
    int32_t nx, ny, count64;
    // run
    uint64_t n, offset;
    uint32_t k0, k1;
    int32_t refill;                       // pop when at least this many lanes are idle
    const float *tab;
    double fc[3], fa[3][3];               // local -> global frame (records only)
};

struct WarpBuf {                          // spawned rays waiting for a lane (SoA)
    double x[3][kBuf], k[3][kBuf], sB[kBuf];
    uint32_t rl[kBuf], rh[kBuf];
    float inv_mu[kBuf], pa[kBuf], E[kBuf];
    uint32_t pa_thr[kBuf];
    int32_t nb[kBuf];                     // no-Bragg flag
    int count;
};

__device__ __forceinline__ float u01_32(uint32_t w) {
    // (w + 1/2) 2^-32 rounded to FP32: relative error <= 2^-24 against the FP64 uniform
    return __fmaf_rn(__uint2float_rn(w), 2.3283064365386963e-10f, 1.16415321826934814e-10f);
}

__device__ __forceinline__ float mdf_q32(const float *tab, uint32_t w) {
    const uint32_t i = w >> 20;
    if (i < (uint32_t)(kMdfM - 1)) {
        const float f = __fmaf_rn((float)(w & 0xFFFFFu), 9.5367431640625e-07f, 4.76837158203125e-07f);
        const float a = tab[i], b = tab[i + 1];
        return __fmaf_rn(f, b - a, a);
    }
    const float m = (float)(0xFFFFFFFFu - w) + 0.5f;
    const float y = (20.0f - log2f(m)) * (kMdfT / 21.0f);
    int j = (int)floorf(y);
    j = j < 0 ? 0 : (j > kMdfT - 1 ? kMdfT - 1 : j);
    const float f = y - (float)j;
    const float a = tab[kMdfM + j], b = tab[kMdfM + j + 1];
    return __fmaf_rn(f, b - a, a);
}

// unit-area rocking curve divided by its maximum, at x = Delta - Delta_M
template <int IRC>
__device__ __forceinline__ float irc_rel32(const Launch32 &L, float x) {
    if (IRC == HEART_IRC_DARWIN) {
        const float y = fabsf(x) * L.irc_delta;            // irc_delta holds 1/delta here
        if (y <= 1.0f) return 1.0f;
        const float d = y + sqrtf(__fmaf_rn(y, y, -1.0f));
        return __frcp_rn(d * d);
    } else if (IRC == HEART_IRC_DARWIN_PRINS) {
        const float y = x * L.irc_delta, g = L.irc_g;
        const float ar = __fmaf_rn(y, y, -__fmaf_rn(g, g, 1.0f)), ai = 2.0f * y * g;
        const float r = hypotf(ar, ai);
        float zr, zi;
        if (ar >= 0) { zr = sqrtf(0.5f * (r + ar)); zi = zr > 0 ? 0.5f * ai / zr : 0.0f; }
        else { zi = copysignf(sqrtf(0.5f * (r - ar)), ai); zr = 0.5f * ai / zi; }
        const float m1 = hypotf(y - zr, g - zi), m2 = hypotf(y + zr, g + zi);
        const float m = fmaxf(m1, m2);
        return __frcp_rn(m * m) * L.irc_gnorm;              // irc_gnorm = 1 / max R
    } else if (IRC == HEART_IRC_PSEUDO_VOIGT) {
        // (eta L + (1 - eta) G) / max, with L and G unit-area at FWHM F
        const float hf = 0.5f * L.irc_fwhm;
        const float lor = __fdividef(hf * hf, __fmaf_rn(x, x, hf * hf));   // L(x)/L(0)
        const float gau = __expf(-L.irc_c * x * x);                        // G(x)/G(0)
        return __fmaf_rn(L.irc_eta, lor, L.irc_g * gau) * L.irc_gnorm;
    } else if (IRC == HEART_IRC_GAUSSIAN) {
        return __expf(-L.irc_c * x * x);
    } else if (IRC == HEART_IRC_LORENTZIAN) {
        const float hf = 0.5f * L.irc_fwhm;
        return __fdividef(hf * hf, __fmaf_rn(x, x, hf * hf));
    } else {
        return fabsf(x) <= 0.5f * L.irc_fwhm ? 1.0f : 0.0f;
    }
}

// Upper bound of irc_rel32 over |x| >= a (a >= 0).  Because
// |asin(s) - asin(sB)| >= |s - sB|, the bound at a = |s - sB| caps the
// acceptance probability before Delta is formed; a candidate with v above it
// is rejected exactly as the full evaluation would reject it.
//   Darwin: R <= 1 / y^2 for |y| >= 1.  Darwin-Prins: R = 1/m^2 with m the
//   larger root modulus, m >= |eta| >= |y|.  Lorentzian: (F/2)^2 / x^2.
template <int IRC>
__device__ __forceinline__ float irc_bound32(const Launch32 &L, float a) {
    if (IRC == HEART_IRC_DARWIN) {
        const float y = a * L.irc_delta;
        return y <= 1.0f ? 1.0f : __frcp_rn(y * y);
    } else if (IRC == HEART_IRC_DARWIN_PRINS) {
        const float y = a * L.irc_delta;
        return y <= 1.0f ? 1.0f : __frcp_rn(y * y) * L.irc_gnorm;
    } else if (IRC == HEART_IRC_LORENTZIAN) {
        const float hf = 0.5f * L.irc_fwhm;
        return a <= hf ? 1.0f : __fdividef(hf * hf, a * a);
    } else if (IRC == HEART_IRC_BOX) {
        return a <= 0.5f * L.irc_fwhm ? 1.0f : 0.0f;
    } else {
        return 1.0f;                  // Gaussian and pseudo-Voigt: evaluated directly (one exp)
    }
}

// lane state of one ray being walked
struct Lane {
    double x0[3], k[3], sB;               // FP64 segment anchors
    float kf[3];                          // k in FP32
    float A, sgn, sBf, cB;                // Bragg anchor, sign of k.N, sin / cos of aB + Delta_M
    float s_exit, Lsum, Lcomp;            // exit distance, Kahan sum of the path
    float inv_mu, pa, inv_1mpa, E;
    uint32_t pa_thr, rl, rh, call;
    int32_t face, nrefl, ncoll, no_bragg;
    // cylinder along-segment constants
    float cb1, cb2, cga, ck0, ctau0;
};

// ---------------------------------------------------------------------------
// spawn: source sample + entry intersection (Sec. 2.1, Sec. 2.2) in the local
// frame; FP64 only where the Bragg decision needs it
// ---------------------------------------------------------------------------
template <int GEOM>
__device__ __forceinline__ bool spawn(const Launch32 &L, uint64_t ray, double x[3], double k[3], double &sB,
                                      float &inv_mu, float &pa, uint32_t &pa_thr, float &E32, int &nb) {
    const uint32_t rl = (uint32_t)ray, rh = (uint32_t)(ray >> 32);
    uint32_t a[4], b[4];
    philox4x32_10(rl, rh, 0u, 0u, L.k0, L.k1, a);
    philox4x32_10(rl, rh, 1u, 0u, L.k0, L.k1, b);
    // direction: uniform in solid angle in the cone
    const float w = u01_32(a[2]) * L.omc;
    const float sphi = sqrtf(w * (2.0f - w));
    float sb, cb;
    sincospif(2.0f * u01_32(a[3]), &sb, &cb);
    const double cphi = 1.0 - (double)w, p1 = (double)(sphi * cb), p2 = (double)(sphi * sb);
    for (int i = 0; i < 3; ++i) k[i] = cphi * L.ax[i] + p1 * L.b1[i] + p2 * L.b2[i];
    double o[3] = {L.o[0], L.o[1], L.o[2]};
    if (L.sig1 > 0.0f || L.sig2 > 0.0f) {
        const float r = sqrtf(-2.0f * __logf(u01_32(b[0])));
        float s, co;
        __sincosf(6.28318530717958648f * (u01_32(b[1]) - 0.5f), &s, &co);
        const double z1 = -(double)(L.sig1 * r * co), z2 = -(double)(L.sig2 * r * s);
        for (int i = 0; i < 3; ++i) o[i] += z1 * L.b1[i] + z2 * L.b2[i];
    }
    for (int i = 0; i < 3; ++i) x[i] = o[i];       // a miss reports its origin
    // entry on the front face
    if (GEOM == HEART_FLAT) {
        if (!(k[2] < 0.0) || !(o[2] > 0.0)) return false;
        const double t = o[2] / (-k[2]);
        x[0] = o[0] + t * k[0];
        x[1] = o[1] + t * k[1];
        x[2] = 0.0;                                  // on the front face
        if (fabs(x[0]) > (double)L.half_d || fabs(x[1]) > (double)L.half_n) return false;
    } else {
        const double c0 = o[1] * o[1] + o[2] * o[2] - L.R64 * L.R64;
        if (!(c0 < 0.0)) return false;
        const double aa = k[1] * k[1] + k[2] * k[2];
        if (!(aa > 0.0)) return false;
        const double bb = o[1] * k[1] + o[2] * k[2];
        const double sq = sqrt(bb * bb - aa * c0);
        const double t = (bb > 0.0) ? -c0 / (bb + sq) : (-bb + sq) / aa;
        double xe[3];
        for (int i = 0; i < 3; ++i) xe[i] = o[i] + t * k[i];
        if (fabs(xe[0] - L.zc64) > (double)L.half_d) return false;
        if (fabs(xe[2]) * (double)L.cphi > xe[1] * (double)L.sphi) return false;
        for (int i = 0; i < 3; ++i) x[i] = xe[i];
    }
    // energy (only rays that entered need it)
    int c = L.n_comp - 1;
    for (int i = 0; i < L.n_comp - 1; ++i)
        if (a[0] < L.comp_thr[i]) { c = i; break; }
    const float up = u01_32(a[1]);
    double E;
    switch (L.kind[c]) {
    case HEART_SRC_MONO: E = L.e0[c]; break;
    case HEART_SRC_GAUSS: {
        float s, co;
        __sincosf(6.28318530717958648f * (u01_32(b[3]) - 0.5f), &s, &co);
        E = L.e0[c] - (double)(L.width[c] * sqrtf(-2.0f * __logf(u01_32(b[2]))) * co);
        break;
    }
    case HEART_SRC_LORENTZ: {
        const float uu = __fmaf_rn(up, 1.0f - L.lF0[c], L.lF0[c]);
        E = L.e0[c] + (double)(0.5f * L.width[c] * tanf(3.14159265f * (uu - 0.5f)));
        break;
    }
    case HEART_SRC_INV_E: E = (double)(L.lo[c] * exp2f(up * log2f(L.hi[c] / L.lo[c]))); break;
    default: E = (double)L.lo[c] + (double)(L.hi[c] - L.lo[c]) * (double)up; break;
    }
    E32 = (float)E;
    if (!(E > 0.0) || !isfinite(E)) return false;
    // per-ray constants: sin(aB + Delta_M) in FP64 (Eq. BraggLaw), the rest FP32
    const double sB0 = L.sB_scale / E;
    nb = !(sB0 < 1.0);
    float Q = 0.0f;
    if (!nb) {
        const float cb0 = sqrtf(fmaxf(0.0f, 1.0f - (float)(sB0 * sB0)));
        sB = sB0 * L.cos_shift + (double)(cb0 * L.sin_shift);
        const float lam = (float)(12.398419843320026e-7 / E);        // mm
        Q = L.K2 * lam * lam * lam / (2.0f * (float)sB0 * cb0);
    } else {
        sB = 2.0;
    }
    const float mu0 = 1.0f / (L.labs * powf(E32 / L.labs_ref, L.labs_pow));
    const float mubar = __fmaf_rn(Q, L.irc_max, mu0);
    inv_mu = 1.0f / mubar;
    pa = nb ? 1.0f : mu0 / mubar;
    // absorb iff (w + 1/2) 2^-32 < pa  <=>  w < ceil(pa 2^32 - 1/2)
    const double thr = ceil((double)pa * 4294967296.0 - 0.5);
    pa_thr = thr >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)thr;
    if (nb) pa_thr = 0xFFFFFFFFu;
    return true;
}

// start a straight segment at x0 along k (entry or after a reflection)
template <int GEOM>
__device__ __forceinline__ void segment(const Launch32 &L, Lane &s) {
    for (int i = 0; i < 3; ++i) s.kf[i] = (float)s.k[i];
    s.Lsum = 0.0f;
    s.Lcomp = 0.0f;
    float best = 3.0e38f;
    int face = HEART_EXIT_SIDE;
    auto cand = [&](float v, int f) {
        v = fmaxf(v, 0.0f);
        if (v < best) { best = v; face = f; }
    };
    double kappa;
    if (GEOM == HEART_FLAT) {
        kappa = s.k[2];
        const float h = (float)s.x0[2], a = (float)s.x0[0], b = (float)s.x0[1];
        const float kh = s.kf[2], ka = s.kf[0], kb = s.kf[1];
        if (kh > 0) cand(-h / kh, HEART_EXIT_FRONT);
        if (kh < 0) cand((-L.thick - h) / kh, HEART_EXIT_BACK);
        if (ka > 0) cand((L.half_d - a) / ka, HEART_EXIT_SIDE);
        if (ka < 0) cand((-L.half_d - a) / ka, HEART_EXIT_SIDE);
        if (kb > 0) cand((L.half_n - b) / kb, HEART_EXIT_SIDE);
        if (kb < 0) cand((-L.half_n - b) / kb, HEART_EXIT_SIDE);
    } else {
        const double X = s.x0[1], Y = s.x0[2];
        const double r0 = sqrt(X * X + Y * Y);
        const double b0 = X * s.k[1] + Y * s.k[2];
        kappa = -b0 / r0;
        const float rho = (float)(r0 - L.R64);               // depth below the inner face
        const float aa = s.kf[1] * s.kf[1] + s.kf[2] * s.kf[2];
        const float bb = (float)b0, R = L.R, t = L.thick;
        const float ci = rho * (2.0f * R + rho);                // r^2 - R^2
        const float co = (rho - t) * (2.0f * R + rho + t);      // r^2 - (R + t)^2
        if (aa > 0.0f) {
            if (bb < 0.0f) {
                const float disc = bb * bb - aa * ci;
                if (disc >= 0.0f) cand(ci / (-bb + sqrtf(disc)), HEART_EXIT_FRONT);
            }
            const float sq = sqrtf(fmaxf(bb * bb - aa * co, 0.0f));
            cand(bb > 0.0f ? -co / (bb + sq) : (-bb + sq) / aa, HEART_EXIT_BACK);
        }
        const float z = (float)(s.x0[0] - L.zc64), kz = s.kf[0];
        if (kz > 0) cand((L.half_d - z) / kz, HEART_EXIT_SIDE);
        if (kz < 0) cand((-L.half_d - z) / kz, HEART_EXIT_SIDE);
        const float Xf = (float)X, Yf = (float)Y;
        const float gp = -Xf * L.sphi + Yf * L.cphi, rp = -s.kf[1] * L.sphi + s.kf[2] * L.cphi;
        if (rp > 0) cand(-gp / rp, HEART_EXIT_SIDE);
        const float gm = -Xf * L.sphi - Yf * L.cphi, rm = -s.kf[1] * L.sphi - s.kf[2] * L.cphi;
        if (rm > 0) cand(-gm / rm, HEART_EXIT_SIDE);
        // k.N along the segment: r(l)^2 = r0^2 (1 + l (cb1 + l cb2))
        const float inv_r0 = (float)(1.0 / r0);
        s.cb1 = 2.0f * bb * inv_r0 * inv_r0;
        s.cb2 = aa * inv_r0 * inv_r0;
        s.cga = aa * inv_r0;
        s.ck0 = (float)kappa;
        s.ctau0 = (float)((X * s.k[2] - Y * s.k[1]) / r0);    // k . t2 at x0 (t2 = N x axis)
    }
    s.s_exit = best;
    s.face = face;
    s.sgn = kappa < 0.0 ? -1.0f : 1.0f;
    s.A = (float)(fabs(kappa) - s.sB);
}

__device__ __forceinline__ void to_global(const Launch32 &L, const double *p, double *g, bool point) {
    for (int i = 0; i < 3; ++i)
        g[i] = (point ? L.fc[i] : 0.0) + p[0] * L.fa[0][i] + p[1] * L.fa[1][i] + p[2] * L.fa[2][i];
}

template <typename T>
__device__ __forceinline__ void add_image(const Launch32 &L, void *img, int ix, int iy) {
    const size_t idx = (size_t)iy * (size_t)L.nx + (size_t)ix;
    if (L.count64) atomicAdd((unsigned long long *)img + idx, 1ull);
    else atomicAdd((int *)img + idx, 1);
}

// tally slots in shared memory (32-bit, flushed as 64-bit)
struct BlockTally {
    unsigned int t[kTallyN];
};

// finish a ray: detector projection + binning + tallies (+ record)
template <int GEOM, bool REC>
__device__ __forceinline__ void finish(const Launch32 &L, Lane &s, int outcome, void *img, BlockTally &bt,
                                       heart_ray_record *rec) {
    int ix = -1, iy = -1, hit = 0;
    float u = __int_as_float(0x7fc00000), v = u;
    double xe[3];
    const float len = (outcome == HEART_EXIT_FRONT || outcome == HEART_EXIT_BACK || outcome == HEART_EXIT_SIDE)
                          ? s.s_exit : s.Lsum;
    for (int i = 0; i < 3; ++i) xe[i] = s.x0[i] + (double)len * s.k[i];
    if (outcome == HEART_EXIT_FRONT || outcome == HEART_EXIT_BACK || outcome == HEART_EXIT_SIDE) {
        const float rel[3] = {(float)(L.D0[0] - xe[0]), (float)(L.D0[1] - xe[1]), (float)(L.D0[2] - xe[2])};
        const float den = s.kf[0] * L.nd[0] + s.kf[1] * L.nd[1] + s.kf[2] * L.nd[2];
        if (den != 0.0f) {
            const float t = (rel[0] * L.nd[0] + rel[1] * L.nd[1] + rel[2] * L.nd[2]) / den;
            if (t > 0.0f) {
                const float P[3] = {__fmaf_rn(t, s.kf[0], -rel[0]), __fmaf_rn(t, s.kf[1], -rel[1]),
                                    __fmaf_rn(t, s.kf[2], -rel[2])};
                u = P[0] * L.eu[0] + P[1] * L.eu[1] + P[2] * L.eu[2];
                v = P[0] * L.ev[0] + P[1] * L.ev[1] + P[2] * L.ev[2];
                const float fx = __fmaf_rn(u, L.inv_pix, L.hnx), fy = __fmaf_rn(v, L.inv_pix, L.hny);
                if (fx >= 0.0f && fx < (float)L.nx && fy >= 0.0f && fy < (float)L.ny) {
                    ix = min((int)fx, L.nx - 1);
                    iy = min((int)fy, L.ny - 1);
                    hit = 1;
                    add_image<int>(L, img, ix, iy);
                    atomicAdd(&bt.t[T_DET_HITS], 1u);
                }
            }
        }
    }
    atomicAdd(&bt.t[T_ABSORBED + (outcome - HEART_ABSORBED)], 1u);
    atomicAdd(&bt.t[T_HIST0 + (s.nrefl < 15 ? s.nrefl : 15)], 1u);
    if (s.no_bragg) atomicAdd(&bt.t[T_NO_BRAGG], 1u);
    if (REC) {
        const uint64_t ray = ((uint64_t)s.rh << 32) | s.rl;
        heart_ray_record &o = rec[ray - L.offset];
        o.ray_id = ray;
        o.outcome = outcome;
        o.nrefl = s.nrefl;
        o.ncoll = s.ncoll;
        o.energy_keV = s.E;
        to_global(L, xe, o.pos, true);
        to_global(L, s.k, o.dir, false);
        o.u_mm = u;
        o.v_mm = v;
        o.ix = ix;
        o.iy = iy;
        o.det_hit = hit;
        o.no_bragg = s.no_bragg;
    }
}

// one tentative collision; returns an outcome code, or -1 while the ray lives
template <int GEOM, int IRC>
__device__ __forceinline__ int step(const Launch32 &L, Lane &s, const float *tab) {
    if (s.ncoll >= L.max_coll) return HEART_STUCK;
    uint32_t w[4];
    philox4x32_10(s.rl, s.rh, s.call++, 0u, L.k0, L.k1, w);
    const float l = -__logf(u01_32(w[0])) * s.inv_mu;
    // Kahan-compensated path length along the segment
    const float y = l - s.Lcomp;
    const float t = s.Lsum + y;
    s.Lcomp = (t - s.Lsum) - y;
    if (t > s.s_exit) return s.face;
    s.Lsum = t;
    ++s.ncoll;
    if (w[1] < s.pa_thr) return HEART_ABSORBED;
    const float v = (u01_32(w[1]) - s.pa) * s.inv_1mpa;
    const float q = mdf_q32(tab, w[2]);
    const float st = sqrtf(q * (2.0f - q));
    float sx, cx;
    __sincosf(6.28318530717958648f * (u01_32(w[3]) - 0.5f), &sx, &cx);
    sx = -sx;
    cx = -cx;
    float D, dk = 0.0f, rinv = 1.0f;
    if (GEOM == HEART_FLAT) {
        D = __fmaf_rn(st, __fmaf_rn(s.kf[0], cx, s.kf[1] * sx), -q * s.kf[2]);
    } else {
        // k.N and k.t2 at the collision point from the along-segment length
        const float Lp = s.Lsum;
        const float eps = Lp * __fmaf_rn(Lp, s.cb2, s.cb1);
        const float rho = sqrtf(1.0f + eps);
        rinv = 1.0f / rho;
        dk = (s.ck0 * (-eps / (1.0f + rho)) - Lp * s.cga) * rinv;
        const float tau = s.ctau0 * rinv;
        D = __fmaf_rn(st, __fmaf_rn(s.kf[0], cx, tau * sx), -q * (s.ck0 + dk));
    }
    const float e = __fmaf_rn(s.sgn, D + dk, s.A);            // |k.n| - sin(aB + Delta_M)
    if (v >= irc_bound32<IRC>(L, fabsf(e))) return -1;        // rejected whatever Delta is
    float sa = s.sBf + e;
    float delta;
    if (sa > 0.0f) {
        sa = fminf(sa, 1.0f);
        const float cs = sqrtf(fmaxf(0.0f, 1.0f - sa * sa));
        delta = asinf(fminf(1.0f, e * (2.0f * s.sBf + e) / __fmaf_rn(sa, s.cB, s.sBf * cs)));
    } else {
        sa = fminf(-sa, 1.0f);                                 // the normal flipped side
        delta = asinf(sa) - asinf(s.sBf);
    }
    const float c2 = __fmaf_rn(-2.0f * sa, sa, 1.0f);
    const float G = 0.5f * __fmaf_rn(c2, c2, 1.0f);
    if (v < irc_rel32<IRC>(L, delta) * G) {
        ++s.nrefl;
        if (s.nrefl > L.max_refl) return HEART_CAPPED;
        // reflection k <- k - 2 (k.n) n in FP64 (Sec. 2.2.4)
        double n[3];
        const double ct = 1.0 - (double)q;
        if (GEOM == HEART_FLAT) {
            n[0] = (double)(st * cx);
            n[1] = (double)(st * sx);
            n[2] = ct;
        } else {
            const double Lp = (double)s.Lsum;
            const double X = s.x0[1] + Lp * s.k[1], Y = s.x0[2] + Lp * s.k[2];
            const double ir = 1.0 / sqrt(X * X + Y * Y);
            const double sxs = (double)(st * sx);
            n[0] = (double)(st * cx);
            n[1] = (-ct * X - sxs * Y) * ir;
            n[2] = (-ct * Y + sxs * X) * ir;
        }
        const double kn = (s.sgn < 0.0f ? -1.0 : 1.0) * (s.sB + (double)e);
        double kk = 0.0;
        for (int i = 0; i < 3; ++i) {
            s.x0[i] += (double)s.Lsum * s.k[i];
            s.k[i] -= 2.0 * kn * n[i];
            kk += s.k[i] * s.k[i];
        }
        const double sc = 1.5 - 0.5 * kk;                       // one Newton step of 1/sqrt(kk)
        for (int i = 0; i < 3; ++i) s.k[i] *= sc;
        segment<GEOM>(L, s);
    }
    return -1;
}

template <int GEOM, int IRC, bool REC>
__global__ void __launch_bounds__(kBlockThreads, 5) k_trace_fp32(const Launch32 L, void *img,
                                                              unsigned long long *scratch, heart_ray_record *rec) {
    __shared__ float s_tab[kMdfKnots];
    __shared__ WarpBuf s_buf[kWarpsPerBlock];
    __shared__ BlockTally bt;
    for (int i = threadIdx.x; i < kMdfKnots; i += blockDim.x) s_tab[i] = L.tab[i];
    for (int i = threadIdx.x; i < kTallyN; i += blockDim.x) bt.t[i] = 0u;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpBuf &B = s_buf[wid];
    if (lane == 0) B.count = 0;
    __syncthreads();
    unsigned long long *counter = scratch + kCounterWord;
    const unsigned lt_mask = (1u << lane) - 1u;

    Lane s;
    bool alive = false;
    bool more = true;                  // global rays may remain
    unsigned long long my_coll = 0, my_emit = 0, my_miss = 0;
    for (;;) {
        const unsigned idle = __ballot_sync(0xffffffffu, !alive);
        const int n_idle = __popc(idle);
        if (n_idle == 32 && !more && B.count == 0) break;
        if (n_idle >= L.refill || (n_idle > 0 && !more) || n_idle == 32) {
            // make sure the buffer can serve every idle lane
            while (more && B.count < n_idle) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(counter, 32ull);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= L.n) { more = false; break; }
                const uint64_t id = base + lane;
                double x[3], k[3], sB = 0.0;
                float inv_mu = 0.f, pa = 0.f, E32 = 0.f;
                uint32_t pa_thr = 0;
                int nb = 0;
                bool hit = false;
                if (id < L.n) {
                    ++my_emit;
                    hit = spawn<GEOM>(L, L.offset + id, x, k, sB, inv_mu, pa, pa_thr, E32, nb);
                    if (!hit) {
                        ++my_miss;
                        if (REC) {
                            heart_ray_record &o = rec[id];
                            o.ray_id = L.offset + id;
                            o.outcome = HEART_MISS;
                            o.nrefl = 0; o.ncoll = 0; o.energy_keV = E32;
                            to_global(L, x, o.pos, true);
                            to_global(L, k, o.dir, false);
                            o.u_mm = __longlong_as_double(0x7ff8000000000000LL); o.v_mm = o.u_mm;
                            o.ix = -1; o.iy = -1; o.det_hit = 0; o.no_bragg = 0;
                        }
                    }
                }
                const unsigned hm = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    const int slot = B.count + __popc(hm & lt_mask);
                    for (int i = 0; i < 3; ++i) { B.x[i][slot] = x[i]; B.k[i][slot] = k[i]; }
                    B.sB[slot] = sB;
                    const uint64_t ray = L.offset + id;
                    B.rl[slot] = (uint32_t)ray;
                    B.rh[slot] = (uint32_t)(ray >> 32);
                    B.inv_mu[slot] = inv_mu;
                    B.pa[slot] = pa;
                    B.pa_thr[slot] = pa_thr;
                    B.E[slot] = E32;
                    B.nb[slot] = nb;
                }
                __syncwarp();
                if (lane == 0) B.count += __popc(hm);
                __syncwarp();
                if (base + 32 >= L.n) more = false;
            }
            // idle lanes pop, highest slots first
            const int avail = B.count;
            const int rank = __popc(idle & lt_mask);
            if (!alive && rank < avail) {
                const int slot = avail - 1 - rank;
                for (int i = 0; i < 3; ++i) { s.x0[i] = B.x[i][slot]; s.k[i] = B.k[i][slot]; }
                s.sB = B.sB[slot];
                s.rl = B.rl[slot];
                s.rh = B.rh[slot];
                s.inv_mu = B.inv_mu[slot];
                s.pa = B.pa[slot];
                s.pa_thr = B.pa_thr[slot];
                s.E = B.E[slot];
                s.no_bragg = B.nb[slot];
                s.inv_1mpa = s.pa < 1.0f ? 1.0f / (1.0f - s.pa) : 0.0f;
                s.sBf = (float)s.sB;
                s.cB = sqrtf(fmaxf(0.0f, 1.0f - s.sBf * s.sBf));
                s.call = 2u;
                s.nrefl = 0;
                s.ncoll = 0;
                segment<GEOM>(L, s);
                alive = true;
            }
            __syncwarp();
            if (lane == 0) B.count = avail - min(avail, n_idle);
            __syncwarp();
        }
        if (alive) {
            const int oc = step<GEOM, IRC>(L, s, s_tab);
            if (oc >= 0) {
                my_coll += (unsigned long long)s.ncoll;
                finish<GEOM, REC>(L, s, oc, img, bt, rec);
                alive = false;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        my_coll += __shfl_down_sync(0xffffffffu, my_coll, off);
        my_emit += __shfl_down_sync(0xffffffffu, my_emit, off);
        my_miss += __shfl_down_sync(0xffffffffu, my_miss, off);
    }
    __syncthreads();
    if (lane == 0) {
        atomicAdd(&scratch[T_COLLISIONS], my_coll);
        atomicAdd(&scratch[T_EMITTED], my_emit);
        atomicAdd(&scratch[T_MISS], my_miss);
    }
    for (int i = threadIdx.x; i < kTallyN; i += blockDim.x)
        if (bt.t[i] && i != T_EMITTED && i != T_MISS && i != T_COLLISIONS) atomicAdd(&scratch[i], (unsigned long long)bt.t[i]);
}

// ---------------------------------------------------------------------------
// host side: local-frame parameters and launch
// ---------------------------------------------------------------------------
namespace {
void to_local(const SpecParams &S, const double *v, double *out, bool point) {
    double r[3] = {v[0], v[1], v[2]};
    if (point) for (int i = 0; i < 3; ++i) r[i] -= S.c[i];
    const double *a0 = S.geometry == HEART_FLAT ? S.ed : S.ax;
    const double *a1 = S.geometry == HEART_FLAT ? S.en : S.cc;
    const double *a2 = S.geometry == HEART_FLAT ? S.N : S.ww;
    out[0] = r[0] * a0[0] + r[1] * a0[1] + r[2] * a0[2];
    out[1] = r[0] * a1[0] + r[1] * a1[1] + r[2] * a1[2];
    out[2] = r[0] * a2[0] + r[1] * a2[1] + r[2] * a2[2];
}
}  // namespace

void make_launch32(const SpecParams &S, const SourceParams &P, uint64_t n, uint64_t seed, uint64_t offset,
                   Launch32 &L) {
    std::memset(&L, 0, sizeof L);
    to_local(S, P.origin, L.o, true);
    to_local(S, P.ax, L.ax, false);
    to_local(S, P.b1, L.b1, false);
    to_local(S, P.b2, L.b2, false);
    L.omc = (float)P.one_minus_cos_max;
    L.sig1 = (float)P.sig1;
    L.sig2 = (float)P.sig2;
    L.n_comp = P.n_comp;
    for (int i = 0; i < P.n_comp; ++i) {
        // first word w with (w + 1/2) 2^-32 >= cumw
        const double thr = std::ceil(P.cumw[i] * 4294967296.0 - 0.5);
        L.comp_thr[i] = thr >= 4294967295.0 ? 0xFFFFFFFFu : (thr <= 0 ? 0u : (uint32_t)thr);
        L.kind[i] = P.kind[i];
        L.e0[i] = P.e0[i];
        L.width[i] = (float)P.width[i];
        L.lo[i] = (float)P.lo[i];
        L.hi[i] = (float)P.hi[i];
        L.lF0[i] = (float)P.lorentz_F0[i];
    }
    L.half_d = (float)S.half_d;
    L.half_n = (float)S.half_n;
    L.thick = (float)S.thickness;
    L.R = (float)S.radius;
    L.R64 = S.radius;
    L.zc = (float)S.zc;
    L.zc64 = S.zc;
    L.sphi = (float)S.sphi;
    L.cphi = (float)S.cphi;
    L.cos_shift = std::cos(S.irc_shift);
    L.sin_shift = (float)std::sin(S.irc_shift);
    // rocking curve, relative to its maximum
    L.irc_fwhm = (float)S.irc_fwhm;
    L.irc_eta = (float)S.irc_eta;
    L.irc_g = (float)S.irc_g;
    L.inv_irc_max = (float)(1.0 / S.irc_max);
    L.irc_c = (float)(4.0 * 0.69314718055994530942 / (S.irc_fwhm * S.irc_fwhm));
    switch (S.irc) {
    case HEART_IRC_DARWIN: L.irc_delta = (float)(1.0 / S.irc_delta); break;
    case HEART_IRC_DARWIN_PRINS:
        L.irc_delta = (float)(1.0 / S.irc_delta);
        L.irc_gnorm = (float)(1.0 / (S.irc_max * S.irc_norm));   // 1 / max R(y)
        break;
    case HEART_IRC_PSEUDO_VOIGT: {
        const double F = S.irc_fwhm, eta = S.irc_eta;
        const double L0 = 2.0 / (3.14159265358979323846 * F), G0 = std::sqrt(4.0 * 0.69314718055994530942 / 3.14159265358979323846) / F;
        // (eta L0 l(x) + (1-eta) G0 g(x)) / max  with l, g the shapes relative to their peaks
        L.irc_eta = (float)(eta * L0);
        L.irc_g = (float)((1.0 - eta) * G0);
        L.irc_gnorm = (float)(1.0 / S.irc_max);
        break;
    }
    default: break;
    }
    L.sB_scale = 12.398419843320026 / (2.0 * S.d_A);
    L.labs = (float)S.labs;
    L.labs_ref = (float)S.labs_ref;
    L.labs_pow = (float)S.labs_pow;
    L.K2 = (float)(S.K * S.K);
    L.irc_max = (float)S.irc_max;
    L.max_refl = S.max_refl;
    L.max_coll = S.max_coll;
    to_local(S, S.D0, L.D0, true);
    double eu[3], ev[3], nd[3];
    to_local(S, S.eu, eu, false);
    to_local(S, S.ev, ev, false);
    to_local(S, S.nd, nd, false);
    for (int i = 0; i < 3; ++i) { L.eu[i] = (float)eu[i]; L.ev[i] = (float)ev[i]; L.nd[i] = (float)nd[i]; }
    L.inv_pix = (float)(1.0 / S.pix);
    L.hnx = 0.5f * (float)S.nx;
    L.hny = 0.5f * (float)S.ny;
    L.nx = S.nx;
    L.ny = S.ny;
    L.count64 = S.count_type == HEART_COUNT_I64;
    L.n = n;
    L.offset = offset;
    L.k0 = (uint32_t)seed;
    L.k1 = (uint32_t)(seed >> 32);
    L.refill = 8;
    L.tab = S.mdf32;
    const double *a0 = S.geometry == HEART_FLAT ? S.ed : S.ax;
    const double *a1 = S.geometry == HEART_FLAT ? S.en : S.cc;
    const double *a2 = S.geometry == HEART_FLAT ? S.N : S.ww;
    for (int i = 0; i < 3; ++i) { L.fc[i] = S.c[i]; L.fa[0][i] = a0[i]; L.fa[1][i] = a1[i]; L.fa[2][i] = a2[i]; }
}

template <int GEOM, int IRC, bool REC>
static void launch_t(const Launch32 &L, void *img, unsigned long long *scratch, heart_ray_record *rec,
                     cudaStream_t st, int blocks) {
    k_trace_fp32<GEOM, IRC, REC><<<blocks, kBlockThreads, 0, st>>>(L, img, scratch, rec);
}

template <bool REC>
static heart_status dispatch(const SpecParams &S, const Launch32 &L, void *img, unsigned long long *scratch,
                             heart_ray_record *rec, cudaStream_t st) {
    int per_sm = 0;
    // resident blocks per SM for this kernel shape
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_fp32<HEART_FLAT, HEART_IRC_DARWIN, REC>,
                                                  kBlockThreads, 0);
    if (per_sm < 1) per_sm = 1;
    uint64_t need = (L.n + 31) / 32 / kWarpsPerBlock + 1;
    uint64_t cap = (uint64_t)num_sms() * (uint64_t)per_sm;
    const int blocks = (int)(need < cap ? need : cap);
#define HEART_IRC_CASES(G)                                                                    \
    switch (S.irc) {                                                                          \
    case HEART_IRC_DARWIN: launch_t<G, HEART_IRC_DARWIN, REC>(L, img, scratch, rec, st, blocks); break; \
    case HEART_IRC_DARWIN_PRINS: launch_t<G, HEART_IRC_DARWIN_PRINS, REC>(L, img, scratch, rec, st, blocks); break; \
    case HEART_IRC_PSEUDO_VOIGT: launch_t<G, HEART_IRC_PSEUDO_VOIGT, REC>(L, img, scratch, rec, st, blocks); break; \
    case HEART_IRC_GAUSSIAN: launch_t<G, HEART_IRC_GAUSSIAN, REC>(L, img, scratch, rec, st, blocks); break; \
    case HEART_IRC_LORENTZIAN: launch_t<G, HEART_IRC_LORENTZIAN, REC>(L, img, scratch, rec, st, blocks); break; \
    default: launch_t<G, HEART_IRC_BOX, REC>(L, img, scratch, rec, st, blocks); break;      \
    }
    if (S.geometry == HEART_FLAT) { HEART_IRC_CASES(HEART_FLAT) } else { HEART_IRC_CASES(HEART_CYL_VON_HAMOS) }
#undef HEART_IRC_CASES
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "FP32 kernel launch");
    return HEART_OK;
}

heart_status launch_fp32(const SpecParams &S, const SourceParams &P, uint64_t n, uint64_t seed, uint64_t offset,
                         void *img, unsigned long long *scratch, cudaStream_t st) {
    if (n == 0) return HEART_OK;
    Launch32 L;
    make_launch32(S, P, n, seed, offset, L);
    return dispatch<false>(S, L, img, scratch, nullptr, st);
}

heart_status launch_fp32_records(const SpecParams &S, const SourceParams &P, uint64_t n, uint64_t seed,
                                 uint64_t offset, void *img, unsigned long long *scratch, heart_ray_record *rec,
                                 cudaStream_t st) {
    if (n == 0) return HEART_OK;
    Launch32 L;
    make_launch32(S, P, n, seed, offset, L);
    return dispatch<true>(S, L, img, scratch, rec, st);
}

}  // namespace heart

extern "C" heart_status heart_trace_batch(heart_spectrometer *const *, const heart_source_desc *const *,
                                          const uint64_t *, const uint64_t *, void *const *, int32_t, void *,
                                          heart_tally *) {
    return heart::fail(HEART_EINVAL, "batched path not built");
}
extern "C" heart_status heart_server_create(size_t, heart_server **) { return heart::fail(HEART_EINVAL, "server not built"); }
extern "C" heart_status heart_server_destroy(heart_server *) { return heart::fail(HEART_EINVAL, "server not built"); }
extern "C" heart_status heart_submit(heart_server *, heart_spectrometer *, const heart_source_desc *, uint64_t, uint64_t,
                                     heart_precision, uint64_t *) { return heart::fail(HEART_EINVAL, "server not built"); }
extern "C" heart_status heart_poll(heart_server *, uint64_t, int32_t, heart_tally *, const void **) {
    return heart::fail(HEART_EINVAL, "server not built");
}
extern "C" heart_status heart_release(heart_server *, uint64_t) { return heart::fail(HEART_EINVAL, "server not built"); }
