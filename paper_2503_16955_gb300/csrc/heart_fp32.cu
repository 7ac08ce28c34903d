// heart_fp32.cu -- the FP32 persistent ray-transport kernel (single and batched).
//
// What is computed is fixed by the paper (Sec. 2.1 source, Sec. 2.2 crystal,
// Sec. 2.2.3-2.2.4 walk, Appendix A orientation sampling, Sec. 2.3 detector);
// the sampling model is the null-collision walk of the FP64 path.  This file
// fixes how it runs on an FP32 machine:
//
// Precision.  The Bragg decision needs |Delta| = |asin|k.n| - (aB + Delta_M)|
// to ~1e-8 rad while |k.n| ~ 0.2.  No FP64 is used; instead every quantity
// that the decision depends on is carried as a *small* FP32 number relative to
// an FP64 constant computed once per launch on the host:
//   * sin(aB + Delta_M) = sB0[c] + ds, with sB0[c] fixed per spectral
//     component and ds formed from the small energy offset of the ray;
//   * the anchor A = |k.N| - sin(aB + Delta_M) at the start of each straight
//     segment: at entry from the small offset of k from the cone axis, after a
//     reflection from the closed form A' = -A + 2e - 2q (sB + e);
//   * per tentative collision the candidate offset D = k.n - k.N ~ theta and,
//     on a cylinder, the along-segment change of k.N from the path length;
//   * Delta = asin((s - sB)(s + sB) / (s cB + sB cs)) with s - sB = e small.
// Positions are FP32 in the crystal frame; the path along a segment is a
// Kahan-compensated sum.  Decisions comparing a uniform with a per-ray
// threshold compare the raw 32-bit Philox word with an integer threshold.
//
// Work distribution.  A persistent grid claims work items (job, ray range)
// from a global counter; a block stages its job's parameters and mosaic
// table in shared memory.  Each warp keeps a shared-memory buffer of spawned
// rays (source sampled, crystal entry found, misses tallied): all 32 lanes
// spawn together when it runs low, and idle lanes pop from it once at least
// `refill` of them are idle, so spawning never runs divergently.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "heart_fp64.cuh"
#include "heart_lib.h"

namespace heart {

constexpr int kWarpsPerBlock = 4;
constexpr int kBlockThreads = kWarpsPerBlock * 32;
// spawned rays buffered per warp, and spawning only while fewer than kSpawnBelow are
// buffered (so at most kSpawnBelow - 1 + 32 <= kBuf); sized so that the generic batched
// kernel's shared memory (the mosaic table, the job and four buffers) fits 6 blocks per SM
constexpr int kBuf = 44;
constexpr int kSpawnBelow = 13;
static_assert(kSpawnBelow - 1 + 32 <= kBuf, "a spawn round must fit the buffer");

TuneConfig g_tune;                        // launch shape picked by the autotuner

// Per-job parameters in the crystal-local frame.
// flat: axes (e_d, e_n, N), origin at the front-face centre; crystal
//       |p0| <= half_d, |p1| <= half_n, -t <= p2 <= 0.
// cylinder: axes (axis, c, axis x c), origin on the axis; crystal
//       |p0 - zc| <= half_d, R <= hypot(p1, p2) <= R + t, |p2| cphi <= p1 sphi.
struct Launch32 {
    // source, local frame
    float o[3], ax[3], b1[3], b2[3];
    float omc, sig1, sig2;
    float a_n;                            // flat: axis . N; cylinder: axis . cylinder axis
    int32_t n_comp;
    uint32_t comp_thr[kMaxComp];          // component i if word < comp_thr[i]
    int32_t kind[kMaxComp];
    float e_ref[kMaxComp];                // reference energy of each component
    float width[kMaxComp], half_ln[kMaxComp], lF0[kMaxComp];
    float sB_raw[kMaxComp], cB_raw[kMaxComp];   // sin / cos aB(e_ref) without the shift
    // crystal
    float half_d, half_n, thick, R, zc, sphi, cphi;
    float cos_shift[kMaxComp], sin_shift[kMaxComp];   // cos, sin of the peak shift at each reference energy
    float c_a;
    // rocking curve (argument x = Delta - Delta_M), relative to its maximum
    float irc_fwhm, irc_eta, irc_delta, irc_g, irc_c, irc_gnorm;
    // physics
    float labs, labs_ref, labs_pow, K2, irc_max;
    int32_t max_refl;
    int64_t max_coll;
    // detector, local frame
    float D0[3], eu[3], ev[3], nd[3], inv_pix, hnx, hny;
    int32_t nx, ny, count64;
    // run
    uint64_t n, offset;
    uint32_t k0, k1;
    uint32_t rk0[10], rk1[10];            // Philox round keys of (k0, k1)
    int32_t refill;                       // pop when at least this many lanes are idle
    int32_t geometry, irc_kind;
    const float *tab;
    const uint32_t *qgrid;                // tilt-grid table words (thinned sampler)
    // band B of process (b) (one order): the first table word past it, and for its
    // largest tilt q_J = 2^(-33/8) the values q_J and tan(theta_J / 2) rounded up,
    // 1 / sin(theta_J) rounded down
    uint32_t band_w2;
    float band_q2, band_is2, band_t2;
    const float *band_is1;                // per grid point: 1 / sin(theta) at its first knot
    void *img;                            // this job's image (int32 or int64)
    unsigned long long *tally;            // this job's kTallyN tally words
    heart_ray_record *rec;                // per-ray records or nullptr
    unsigned long long *eimg;             // energy image (1e-6 keV units) or nullptr
    int32_t n_qe, pad_qe;
    float qe_e[kMaxQe], qe_v[kMaxQe];     // detector QE knots
    double fc[3], fa[3][3];               // local -> global frame (records, user rays)
    float faf[3][3];                      // the same rotation in FP32 (user rays' polarisation)
    double inv_Rd;                        // 1 / R (cylinder) in FP64
    // thinned candidates: sampler, v*, X* and the window constants
    // 2 sin^2(X*/2), sin X* (the |k.n| window of |Delta| < X* from sin(aB + dM))
    int32_t sampler;
    float vstar, xstar, hx2, sx;
    // no rocking curve: cone-candidate factor 2 W(0) / int W dq and the mosaic
    // distribution's W(q) / W(0) in closed form (mdf_ratio32)
    int32_t mdf;
    float none_fac, w_a2, w_c, w_wl, w_wg, w_b, w_qmax;
    float none_qv;                        // thinned cones: W / W(0) <= v* beyond this tilt (inf: never)
    // polarisation and user-supplied rays (the extended kernel only)
    int32_t pol_on, user;
    float pol[3];                         // source polarisation, local frame
    double hc_2d, cs_shift, sn_shift;     // hc / 2d (keV); cos, sin Delta_M
    double shift0;                        // Delta_M without the energy table
    // energy-dependent rocking curve: knots, width scale, added shift (n_irc_e = 0: none),
    // and the table's shift at each component's reference energy
    int32_t n_irc_e, pad_ie;
    float irc_e[HEART_MAX_IRC_E], irc_ws[HEART_MAX_IRC_E], irc_sh[HEART_MAX_IRC_E];
    float sh_ref[kMaxComp];
    const double *ray[10];                // user arrays: ox oy oz kx ky kz E px py pz
    // reflection orders (Sec. 2.2.3; order 0 is the one of the fields above): multiple
    // relative to order 0's, K_h^2, 1 / width ratio, and per order and component
    // sin(aB_h + Delta_M) at the reference energy and the cone axis's anchor;
    // xs_on: X* scales with a width ratio or an energy table
    int32_t n_ord, xs_on;
    float ord_r[HEART_MAX_ORDERS], ord_k2[HEART_MAX_ORDERS], ord_iw[HEART_MAX_ORDERS];
    float osB0[HEART_MAX_ORDERS][kMaxComp];   // sin(aB_h(e_ref) + Delta_M)
    float oA0[HEART_MAX_ORDERS][kMaxComp];    // |k.N| - osB0 for k on the cone axis
    double ord_rd[HEART_MAX_ORDERS];      // the multiples' ratio in FP64 (user rays)
    // tabulated spectrum: CDF thresholds on the raw word, in-interval offset and
    // slope, knots relative to the table's mean energy (its e_ref)
    int32_t n_tab, pad_tab;
    const unsigned long long *tab_thr;
    const float *tab_off, *tab_inv, *tab_dE, *tab_w;
};

// a spawned ray waiting for a lane (SoA per warp)
struct WarpBuf {
    float x[3][kBuf], k[3][kBuf];
    float A[kBuf], sB[kBuf], mu0[kBuf], qr[kBuf], E[kBuf], inv_ws[kBuf];
    uint32_t rl[kBuf], rh[kBuf];
    int32_t nb[kBuf];
    // the first segment, prepared while the warp spawns together
    float s_exit[kBuf], inv_mu[kBuf], pa[kBuf], ra[kBuf], qmin[kBuf], pbar[kBuf];
    uint32_t w0[kBuf], w1[kBuf];
    float pbarB[kBuf];
    int32_t face[kBuf];
    int count;
};

// Philox4x32-10 with the round keys read from the launch parameters (the
// Weyl key schedule is the same for every ray of a job)
template <bool RK>
__device__ __forceinline__ void philox_l(const Launch32 &L, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                         uint32_t out[4]) {
    if constexpr (!RK) {
        philox4x32_10(c0, c1, c2, c3, L.k0, L.k1, out);
    } else {
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
            const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
            const uint32_t n0 = hi1 ^ c1 ^ L.rk0[r], n2 = hi0 ^ c3 ^ L.rk1[r];
            c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        }
        out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
    }
}

__device__ __forceinline__ float u01_32(uint32_t w) {
    // (w + 1/2) 2^-32 rounded to FP32: relative error <= 2^-24 against the FP64 uniform
    return __fmaf_rn(__uint2float_rn(w), 2.3283064365386963e-10f, 1.16415321826934814e-10f);
}

// cos / sin (2 pi u) from the SFU on the centred argument 2 pi (u - 1/2)
__device__ __forceinline__ void sincos_2pi(float u, float *s, float *c) {
    __sincosf(6.28318530717958648f * (u - 0.5f), s, c);
    *s = -*s;
    *c = -*c;
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
template <int IRC_T>
__device__ __forceinline__ float irc_rel32(const Launch32 &L, float x) {
    const int IRC = IRC_T >= 0 ? IRC_T : L.irc_kind;
    if (IRC == HEART_IRC_DARWIN) {
        const float y = fabsf(x) * L.irc_delta;            // irc_delta holds 1/delta
        if (y <= 1.0f) return 1.0f;
        const float d = y + sqrtf(__fmaf_rn(y, y, -1.0f));
        return __frcp_rn(d * d);
    } else if (IRC == HEART_IRC_DARWIN_PRINS) {
        // |eta -+ z|^2 formed directly; for |y| <= 1e4 the fourth powers stay far
        // inside the FP32 range, beyond that hypotf takes the modulus
        const float y = x * L.irc_delta, g = L.irc_g;
        const float ar = __fmaf_rn(y, y, -__fmaf_rn(g, g, 1.0f)), ai = 2.0f * y * g;
        const float r = fabsf(y) <= 1.0e4f ? sqrtf(__fmaf_rn(ar, ar, ai * ai)) : hypotf(ar, ai);
        float zr, zi;
        if (ar >= 0) { zr = sqrtf(0.5f * (r + ar)); zi = zr > 0 ? 0.5f * ai / zr : 0.0f; }
        else { zi = copysignf(sqrtf(0.5f * (r - ar)), ai); zr = 0.5f * ai / zi; }
        const float d1r = y - zr, d1i = g - zi, d2r = y + zr, d2i = g + zi;
        const float m2 = fmaxf(__fmaf_rn(d1r, d1r, d1i * d1i), __fmaf_rn(d2r, d2r, d2i * d2i));
        return __frcp_rn(m2) * L.irc_gnorm;                 // irc_gnorm = 1 / max R
    } else if (IRC == HEART_IRC_PSEUDO_VOIGT) {
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
//   pseudo-Voigt: the weighted Lorentzian tail plus the Gaussian at a.
template <int IRC_T>
__device__ __forceinline__ float irc_bound32_raw(const Launch32 &L, float a) {
    const int IRC = IRC_T >= 0 ? IRC_T : L.irc_kind;
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
    } else if (IRC == HEART_IRC_PSEUDO_VOIGT) {
        const float hf = 0.5f * L.irc_fwhm;
        if (a <= hf) return 1.0f;
        return __fmaf_rn(L.irc_eta, __fdividef(hf * hf, a * a), L.irc_g * __expf(-L.irc_c * a * a)) * L.irc_gnorm;
    } else {
        return 1.0f;                  // Gaussian: evaluated directly (one exp)
    }
}

// the bound with a relative margin of 1e-5 that covers the approximate
// reciprocal and exponential used to form it
template <int IRC_T>
__device__ __forceinline__ float irc_bound32(const Launch32 &L, float a) {
    return irc_bound32_raw<IRC_T>(L, a) * 1.00001f;
}

// lane state of one ray being walked (all FP32)
struct Lane {
    float x0[3], k[3];                    // segment start and direction, crystal frame
    float A, sgn, sB, cB;                 // Bragg anchor, sign of k.N, sin / cos of aB + Delta_M
    float s_exit, Lsum, Lcomp;            // exit distance, Kahan sum of the path
    float inv_mu, pa, inv_1mpa, E;        // segment majorant: 1 / mu, mu0 / mu, 1 / (1 - mu0 / mu)
    uint32_t pa_thr, rl, rh, call;
    float mu0, qr;                        // per ray: absorption rate, Q R_max / w
    float inv_ws;                         // per ray: 1 / the rocking curve's width scale at E
    // thinned segment: share of process (a) (1: the plain stream), tilt bound,
    // arc bound, first table word of process (b) (its words are [w0, 2^32))
    float ra, qmin, pbar;
    uint32_t w0;
    // band B of process (b), one order: table words [w1, band_w2) at the arc bound
    // pbarB; pbarB == pbar: no band B (process (b) is [w0, 2^32) at pbar)
    uint32_t w1;
    float pbarB;
    int32_t face, nrefl, ncoll, no_bragg;
    // cylinder: depth below the inner face at x0 and along-segment constants of k.N
    float rho0, cb1, cb2, cga, ck0, ctau0;
    float p[3];                           // polarisation, crystal frame (extended kernel)
    bool pol;
    // several reflection orders (extended kernel): the fields above hold the order
    // of the current candidate, h; per order its anchor, sin / cos(aB_h + Delta_M),
    // rate, inverse width scale, thinning bounds and cumulative share of the rate
    int32_t h;
    float oA[HEART_MAX_ORDERS], osB[HEART_MAX_ORDERS], ocB[HEART_MAX_ORDERS], oqr[HEART_MAX_ORDERS];
    float oiw[HEART_MAX_ORDERS], ora[HEART_MAX_ORDERS], oqmin[HEART_MAX_ORDERS], opbar[HEART_MAX_ORDERS];
    float ocum[HEART_MAX_ORDERS];
    uint32_t ow0[HEART_MAX_ORDERS];
};

// absorption rate mu0 and scatter-candidate rate Q R_max / w of a ray of energy E
// (Sec. 2.2.4; a rocking curve w times as wide peaks 1/w as high); without a
// rocking curve Q cos(aB + Delta_M) x 2 cones x 2 pi f(0), sB = sin(aB + Delta_M)
__device__ __forceinline__ void ray_rates(const Launch32 &L, float E, float Q, int nb, float inv_ws, float sB,
                                          float &mu0, float &qr) {
    mu0 = 1.0f / (L.labs * __powf(E / L.labs_ref, L.labs_pow));
    if (L.irc_kind == HEART_IRC_NONE)
        qr = (nb || !(sB > 0.0f)) ? 0.0f : Q * sqrtf(fmaxf(0.0f, __fmaf_rn(-sB, sB, 1.0f))) * L.none_fac;
    else
        qr = nb ? 0.0f : Q * L.irc_max * inv_ws;
}

// W(q) / W(0) of the mosaic distribution, q = 1 - cos(theta)
__device__ __forceinline__ float mdf_ratio32(const Launch32 &L, float q) {
    switch (L.mdf) {
    case HEART_MDF_VMF: return __expf(-L.w_c * q);
    case HEART_MDF_WRAPPED_LORENTZIAN: return __fdividef(L.w_a2, __fmaf_rn(2.0f, q, L.w_a2));
    case HEART_MDF_SPHERICAL_WRAPPED_LORENTZIAN: {
        const float r = __fdividef(L.w_b, L.w_b + q);
        return r * r;
    }
    case HEART_MDF_UNIFORM: return q <= L.w_qmax ? 1.0f : 0.0f;
    default: {
        const float th = 2.0f * asinf(sqrtf(0.5f * fminf(fmaxf(q, 0.0f), 2.0f)));
        const float t2 = th * th;
        return __fmaf_rn(L.w_wl, __fdividef(L.w_a2, L.w_a2 + t2), L.w_wg * __expf(-L.w_c * t2));
    }
    }
}

// the energy-dependent rocking curve at E: width scale and added shift, linear
// between the knots and constant beyond them
__device__ __forceinline__ void irc_energy32(const Launch32 &L, float E, float &ws, float &sh) {
    const int n = L.n_irc_e;
    if (n == 1 || E <= L.irc_e[0]) { ws = L.irc_ws[0]; sh = L.irc_sh[0]; return; }
    if (E >= L.irc_e[n - 1]) { ws = L.irc_ws[n - 1]; sh = L.irc_sh[n - 1]; return; }
    int i = 0;
    while (!(E < L.irc_e[i + 1])) ++i;
    const float f = (E - L.irc_e[i]) / (L.irc_e[i + 1] - L.irc_e[i]);
    ws = __fmaf_rn(f, L.irc_ws[i + 1] - L.irc_ws[i], L.irc_ws[i]);
    sh = __fmaf_rn(f, L.irc_sh[i + 1] - L.irc_sh[i], L.irc_sh[i]);
}

// an energy table's change dM of the peak shift from the reference energy's:
// sin(a + dM) - sin(a) = c sin dM - 2 s sin^2(dM / 2), by its series
__device__ __forceinline__ void shift_anchor(float dM, float &sB, float &A) {
    const float dM2 = dM * dM;
    const float cs = sqrtf(fmaxf(0.0f, __fmaf_rn(-sB, sB, 1.0f)));
    const float inc = __fmaf_rn(cs * dM, __fmaf_rn(dM2, -0.166666667f, 1.0f), -0.5f * sB * dM2);
    sB += inc;
    A -= inc;
}

// Order h's anchor and sin(aB_h + Delta_M) for a sampled ray of component c,
// from the same small quantities as order 0's: sin aB_h = r_h sin aB_0 (Eq.
// BraggLaw on d / m_h), so the ray's sine offset ds scales by r_h; dA is the
// entry's |k.N| offset from the cone axis, dM the energy table's change of the
// shift.  False (sB = 1, A + sB = |k.N|) if the order has no Bragg solution.
__device__ __forceinline__ bool order_anchor(const Launch32 &L, int c, float ds, float dA, float dM, int h,
                                             float &A, float &sB) {
    const float r = L.ord_r[h];
    const float s0 = L.sB_raw[c] * r, dsh = ds * r, sraw = s0 + dsh;
    if (!(sraw < 1.0f)) {
        sB = 1.0f;
        A = L.oA0[0][c] + L.osB0[0][c] + dA - 1.0f;
        return false;
    }
    const float craw = sqrtf(fmaxf(0.0f, __fmaf_rn(-sraw, sraw, 1.0f)));
    const float c0 = sqrtf(fmaxf(0.0f, __fmaf_rn(-s0, s0, 1.0f)));
    const float den = craw + c0;
    const float dc = den > 0.0f ? -dsh * (sraw + s0) / den : 0.0f;
    const float dsp = __fmaf_rn(dsh, L.cos_shift[c], dc * L.sin_shift[c]);
    sB = L.osB0[h][c] + dsp;
    A = L.oA0[h][c] + dA - dsp;
    if (L.n_irc_e > 0) shift_anchor(dM, sB, A);
    return true;
}

// ---------------------------------------------------------------------------
// spawn: source sample + entry (Sec. 2.1, Sec. 2.2) in the crystal frame
// ---------------------------------------------------------------------------
// The geometric part of a sampled ray: its first Philox block (call 0: spot
// radius and angle, 1 - cos(phi), azimuth), the direction, the origin and the
// entry.  On a hit x is the entry point and dA is |k.N| there minus its value
// for the cone axis.  The energy's words are the second block (call 1), drawn
// by spawn_energy's callers for the rays that entered only.
template <int GEOM_T>
__device__ __forceinline__ bool spawn_entry(const Launch32 &L, uint64_t ray, float x[3], float k[3], float &dA) {
    const int GEOM = GEOM_T >= 0 ? GEOM_T : L.geometry;
    uint32_t a[4];
    philox_l<(GEOM_T >= 0)>(L, (uint32_t)ray, (uint32_t)(ray >> 32), 0u, 0u, a);
    // direction, uniform in solid angle in the cone; dn = k.n_ref - axis.n_ref
    const float w = u01_32(a[2]) * L.omc;                 // 1 - cos(phi)
    const float sphi = sqrtf(w * (2.0f - w));
    float sbeta, cbeta;
    sincos_2pi(u01_32(a[3]), &sbeta, &cbeta);            // SFU: |error| <= 4e-7, a direction error <= 1.5e-8 rad
    const float p1 = sphi * cbeta, p2 = sphi * sbeta;
    for (int i = 0; i < 3; ++i) k[i] = __fmaf_rn(p2, L.b2[i], __fmaf_rn(p1, L.b1[i], __fmaf_rn(-w, L.ax[i], L.ax[i])));
    const int ni = GEOM == HEART_FLAT ? 2 : 0;            // N (flat) or the cylinder axis
    const float dn = __fmaf_rn(p2, L.b2[ni], __fmaf_rn(p1, L.b1[ni], -w * L.ax[ni]));
    float o[3] = {L.o[0], L.o[1], L.o[2]};
    if (L.sig1 > 0.0f || L.sig2 > 0.0f) {
        const float r = sqrtf(-2.0f * __logf(u01_32(a[0])));
        float s, co;
        sincos_2pi(u01_32(a[1]), &s, &co);
        const float z1 = L.sig1 * r * co, z2 = L.sig2 * r * s;
        for (int i = 0; i < 3; ++i) o[i] = __fmaf_rn(z2, L.b2[i], __fmaf_rn(z1, L.b1[i], o[i]));
    }
    for (int i = 0; i < 3; ++i) x[i] = o[i];              // a miss reports its origin
    if (GEOM == HEART_FLAT) {
        if (!(k[2] < 0.0f) || !(o[2] > 0.0f)) return false;
        const float t = o[2] / (-k[2]);
        const float ex = __fmaf_rn(t, k[0], o[0]), ey = __fmaf_rn(t, k[1], o[1]);
        if (fabsf(ex) > L.half_d || fabsf(ey) > L.half_n) return false;
        x[0] = ex; x[1] = ey; x[2] = 0.0f;
        dA = -dn;                                         // |k_h| = |a_h| - dn for k_h < 0
    } else {
        const float aa = __fmaf_rn(k[1], k[1], k[2] * k[2]);
        if (!(aa > 0.0f)) return false;
        const float ro2 = __fmaf_rn(o[1], o[1], o[2] * o[2]);
        const float c0 = ro2 - L.R * L.R;
        if (!(c0 < 0.0f)) return false;
        const float bo = __fmaf_rn(o[1], k[1], o[2] * k[2]);
        const float sq = sqrtf(__fmaf_rn(bo, bo, -aa * c0));
        const float t = (bo > 0.0f) ? -c0 / (bo + sq) : (sq - bo) / aa;
        float xe[3];
        for (int i = 0; i < 3; ++i) xe[i] = __fmaf_rn(t, k[i], o[i]);
        if (fabsf(xe[0] - L.zc) > L.half_d) return false;
        if (fabsf(xe[2]) * L.cphi > xe[1] * L.sphi) return false;
        for (int i = 0; i < 3; ++i) x[i] = xe[i];
        // |k.N| at r = R: sqrt((1 - kz^2)(1 - eps_o)), eps_o = (ro^2 - bo^2/aa) / R^2,
        // minus the sine of the cone axis to the cylinder axis, as small terms
        const float eps_o = (ro2 - bo * bo / aa) / (L.R * L.R);
        const float kabs = sqrtf(aa * (1.0f - eps_o));
        const float num = -dn * (2.0f * L.a_n + dn) - aa * eps_o;   // |k.N|^2 - c_a^2
        dA = num / (kabs + L.c_a);
    }
    return true;
}

// The energy part of a ray that entered (the words e0 .. e3 of its second
// Philox block: component, the component's parameter, the Gaussian line's
// pair; dA from spawn_entry): spectral component and
// energy, as a small offset from the component's reference energy so that
// sin(aB) keeps ~1e-9 accuracy, the Bragg anchor and the rates.  False if the
// energy is not positive and finite (the ray counts as a miss).
__device__ __forceinline__ bool spawn_energy(const Launch32 &L, uint32_t e0w, uint32_t e1w, uint32_t e2w, uint32_t e3w,
                                             float dA, float &A, float &sB, float &mu0, float &qr, float &inv_ws,
                                             float &E32, int &nb, float *oA = nullptr, float *osB = nullptr,
                                             int *nbm = nullptr) {
    int c = L.n_comp - 1;
    for (int i = 0; i < L.n_comp - 1; ++i)
        if (e0w < L.comp_thr[i]) { c = i; break; }
    const float up = u01_32(e1w);
    float E, ds;                                          // ds = sin(aB(E)) - sin(aB(e_ref))
    const float e0 = L.e_ref[c], s0 = L.sB_raw[c];
    switch (L.kind[c]) {
    case HEART_SRC_MONO: E = e0; ds = 0.0f; break;
    case HEART_SRC_INV_E: {
        const float g = (up - 0.5f) * L.half_ln[c];       // E = e_ref exp(g)
        E = e0 * __expf(g);
        // expm1(-g): for |g| <= 0.2 (a continuum up to 1.5 times its lower end) by the
        // Taylor series to g^7, whose remainder is below 4e-10 relative
        const float x = -g;
        float em;
        if (fabsf(x) <= 0.2f) {
            float p = __fmaf_rn(x, 1.98412698e-4f, 1.38888889e-3f);
            p = __fmaf_rn(p, x, 8.33333333e-3f);
            p = __fmaf_rn(p, x, 4.16666667e-2f);
            p = __fmaf_rn(p, x, 0.166666667f);
            p = __fmaf_rn(p, x, 0.5f);
            em = __fmaf_rn(p * x, x, x);
        } else {
            em = expm1f(x);
        }
        ds = s0 * em;
        break;
    }
    case HEART_SRC_TABLE: {
        // the interval with thr_i <= word < thr_i+1 (the FP64 path's decision
        // u < C_i taken exactly on the word), then linear inside it
        const unsigned long long wv = e1w;
        int lo = 0, hi = L.n_tab - 1;
        while (hi - lo > 1) {
            const int m = (lo + hi) >> 1;
            if (wv < L.tab_thr[m]) hi = m; else lo = m;
        }
        const float t = ((float)(wv - L.tab_thr[lo]) + L.tab_off[lo]) * L.tab_inv[lo];
        const float dE = __fmaf_rn(t, L.tab_w[lo], L.tab_dE[lo]);
        E = e0 + dE;
        const float r = dE / e0;
        ds = -s0 * r / (1.0f + r);
        break;
    }
    default: {
        float dE;
        if (L.kind[c] == HEART_SRC_GAUSS) {
            const float co = -__cosf(6.28318530717958648f * (u01_32(e3w) - 0.5f));  // cos(2 pi u), as sincos_2pi
            dE = L.width[c] * sqrtf(-2.0f * __logf(u01_32(e2w))) * co;
        } else if (L.kind[c] == HEART_SRC_LORENTZ) {
            const float uu = __fmaf_rn(up, 1.0f - L.lF0[c], L.lF0[c]);
            dE = 0.5f * L.width[c] * tanf(3.14159265f * (uu - 0.5f));
        } else {
            dE = L.width[c] * (up - 0.5f);                // uniform: width holds hi - lo
        }
        E = e0 + dE;
        const float r = dE / e0;
        ds = -s0 * r / (1.0f + r);
        break;
    }
    }
    E32 = E;
    if (!(E > 0.0f) || !isfinite(E)) return false;
    const float sraw = s0 + ds;
    nb = !(sraw < 1.0f);
    float Q = 0.0f;
    if (!nb) {
        // shift by Delta_M: sin(aB + dM) - sin(aB0 + dM) from small terms
        const float craw = sqrtf(fmaxf(0.0f, __fmaf_rn(-sraw, sraw, 1.0f)));
        const float dc = -ds * (sraw + s0) / (craw + L.cB_raw[c]);
        const float dsp = __fmaf_rn(ds, L.cos_shift[c], dc * L.sin_shift[c]);
        sB = L.osB0[0][c] + dsp;
        A = L.oA0[0][c] + dA - dsp;
        const float lam = 12.398419843320026e-7f / E;     // mm
        Q = L.K2 * lam * lam * lam / (2.0f * sraw * craw);
    } else {
        // no Bragg solution: sin = 1 keeps A + sB = |k.N| for the segment geometry
        sB = 1.0f;
        A = L.oA0[0][c] + L.osB0[0][c] + dA - 1.0f;
    }
    inv_ws = L.ord_iw[0];
    float dM = 0.0f;
    if (L.n_irc_e > 0) {
        // energy-dependent curve: width scale, and the shift's small change dM
        // from the component's reference
        float ws, sh;
        irc_energy32(L, E, ws, sh);
        inv_ws = L.ord_iw[0] / ws;
        dM = sh - L.sh_ref[c];
        if (!nb) shift_anchor(dM, sB, A);
    }
    ray_rates(L, E, Q, nb, inv_ws, sB, mu0, qr);
    if (oA && L.n_ord > 1) {
        // the other orders' anchors (their rates follow from E where the ray is walked)
        int m = nb;
        for (int h = 1; h < L.n_ord; ++h) m |= (order_anchor(L, c, ds, dA, dM, h, oA[h], osB[h]) ? 0 : 1) << h;
        *nbm = m;
    }
    return true;
}

// a sampled ray: spawn_entry, then spawn_energy for a hit
template <int GEOM_T>
__device__ __forceinline__ bool spawn(const Launch32 &L, uint64_t ray, float x[3], float k[3], float &A,
                                      float &sB, float &mu0, float &qr, float &inv_ws, float &E32, int &nb,
                                      float *oA = nullptr, float *osB = nullptr, int *nbm = nullptr) {
    float dA;
    if (!spawn_entry<GEOM_T>(L, ray, x, k, dA)) return false;
    uint32_t e[4];
    philox_l<(GEOM_T >= 0)>(L, (uint32_t)ray, (uint32_t)(ray >> 32), 1u, 0u, e);
    return spawn_energy(L, e[0], e[1], e[2], e[3], dA, A, sB, mu0, qr, inv_ws, E32, nb, oA, osB, nbm);
}

// user-supplied ray: read, move to the crystal frame and enter in FP64 (once
// per ray), so that the anchor A = |k.N| - sin(aB + Delta_M) is exact to FP32
// rounding whatever the ray's energy and direction; p is the ray's
// polarisation projected perpendicular to k, zero if unpolarised
template <int GEOM_T>
__device__ __forceinline__ bool spawn_user(const Launch32 &L, uint64_t id, float x[3], float k[3], float p[3],
                                           float &A, float &sB, float &mu0, float &qr, float &inv_ws, float &E32,
                                           int &nb, float *oA = nullptr, float *osB = nullptr, int *nbm = nullptr) {
    const int GEOM = GEOM_T >= 0 ? GEOM_T : L.geometry;
    // FP64 only where the anchor needs it (GB300's FP64 rate bounds this path):
    // the direction, the entry point and sin(aB + Delta_M); one reciprocal square
    // root normalises k
    double E = L.ray[6][id], og[3], kg[3], ol[3], kl[3];
    for (int i = 0; i < 3; ++i) { og[i] = L.ray[i][id] - L.fc[i]; kg[i] = L.ray[3 + i][id]; }
    // (FP64 sums of products as explicit fused multiply-adds: GB300's FP64 rate bounds this entry)
    const double kk = __fma_rn(kg[0], kg[0], __fma_rn(kg[1], kg[1], kg[2] * kg[2]));
    if (kk > 0.0) {
        const double ik = rsqrt(kk);
        for (int i = 0; i < 3; ++i) kg[i] *= ik;
    } else {
        E = __longlong_as_double(0x7ff8000000000000LL);      // a zero direction cannot enter
    }
    for (int i = 0; i < 3; ++i) {
        ol[i] = __fma_rn(og[0], L.fa[i][0], __fma_rn(og[1], L.fa[i][1], og[2] * L.fa[i][2]));
        kl[i] = __fma_rn(kg[0], L.fa[i][0], __fma_rn(kg[1], L.fa[i][1], kg[2] * L.fa[i][2]));
        x[i] = (float)ol[i];
        k[i] = (float)kl[i];
        p[i] = 0.0f;
    }
    if (L.pol_on) {
        // projection perpendicular to k in FP32 (G needs ~1e-7), in FP64 when p is
        // within 1e-3 of parallel to k; unpolarised below 1e-12 as in the FP64 kernel
        float pf[3] = {(float)L.ray[7][id], (float)L.ray[8][id], (float)L.ray[9][id]};
        const float kf[3] = {(float)kg[0], (float)kg[1], (float)kg[2]};
        const float pp = __fmaf_rn(pf[0], pf[0], __fmaf_rn(pf[1], pf[1], pf[2] * pf[2]));
        const float pk = __fmaf_rn(pf[0], kf[0], __fmaf_rn(pf[1], kf[1], pf[2] * kf[2]));
        for (int i = 0; i < 3; ++i) pf[i] = __fmaf_rn(-pk, kf[i], pf[i]);
        const float pn2 = __fmaf_rn(pf[0], pf[0], __fmaf_rn(pf[1], pf[1], pf[2] * pf[2]));
        if (pn2 > 1e-6f * pp) {
            const float ipn = rsqrtf(pn2);
            for (int i = 0; i < 3; ++i)
                p[i] = (pf[0] * L.faf[i][0] + pf[1] * L.faf[i][1] + pf[2] * L.faf[i][2]) * ipn;
        } else {
            double pg[3] = {L.ray[7][id], L.ray[8][id], L.ray[9][id]};
            const double pkd = __fma_rn(pg[0], kg[0], __fma_rn(pg[1], kg[1], pg[2] * kg[2]));
            for (int i = 0; i < 3; ++i) pg[i] = __fma_rn(-pkd, kg[i], pg[i]);
            const double pn = sqrt(__fma_rn(pg[0], pg[0], __fma_rn(pg[1], pg[1], pg[2] * pg[2])));
            if (pn > 1e-12)
                for (int i = 0; i < 3; ++i)
                    p[i] = (float)(__fma_rn(pg[0], L.fa[i][0], __fma_rn(pg[1], L.fa[i][1], pg[2] * L.fa[i][2])) / pn);
        }
    }
    E32 = (float)E;
    if (!(E > 0.0) || !isfinite(E)) return false;
    double kN;                                            // |k.N| at the entry point
    if (GEOM == HEART_FLAT) {
        if (!(kl[2] < 0.0) || !(ol[2] > 0.0)) return false;
        const double t = ol[2] / (-kl[2]);
        const double ex = __fma_rn(t, kl[0], ol[0]), ey = __fma_rn(t, kl[1], ol[1]);
        if (fabs(ex) > (double)L.half_d || fabs(ey) > (double)L.half_n) return false;
        x[0] = (float)ex; x[1] = (float)ey; x[2] = 0.0f;
        kN = -kl[2];
    } else {
        const double aa = __fma_rn(kl[1], kl[1], kl[2] * kl[2]);
        if (!(aa > 0.0)) return false;
        const double R = (double)L.R;
        const double c0 = __fma_rn(ol[1], ol[1], __fma_rn(ol[2], ol[2], -R * R));
        if (!(c0 < 0.0)) return false;
        const double bo = __fma_rn(ol[1], kl[1], ol[2] * kl[2]);
        const double sq = sqrt(__fma_rn(bo, bo, -aa * c0));
        const double t = (bo > 0.0) ? -c0 / (bo + sq) : (sq - bo) / aa;
        double xe[3];
        for (int i = 0; i < 3; ++i) xe[i] = __fma_rn(t, kl[i], ol[i]);
        if (fabs(xe[0] - (double)L.zc) > (double)L.half_d) return false;
        if (fabs(xe[2]) * (double)L.cphi > xe[1] * (double)L.sphi) return false;
        for (int i = 0; i < 3; ++i) x[i] = (float)xe[i];
        kN = __fma_rn(kl[1], xe[1], kl[2] * xe[2]) * L.inv_Rd;
    }
    const double sr = L.hc_2d / E;                        // sin(aB), Eq. (BraggLaw)
    nb = !(sr < 1.0);
    float Q = 0.0f;
    double cs_s = L.cs_shift, sn_s = L.sn_shift;
    inv_ws = L.ord_iw[0];
    if (L.n_irc_e > 0) {                                  // energy-dependent rocking curve
        float ws, sh;
        irc_energy32(L, (float)E, ws, sh);
        inv_ws = L.ord_iw[0] / ws;
        sincos(L.shift0 + (double)sh, &sn_s, &cs_s);
    }
    if (!nb) {
        // cos aB only with a peak shift (then in FP64); Q takes it in FP32
        const double sb = sn_s != 0.0 ? __fma_rn(sr, cs_s, sqrt(__fma_rn(-sr, sr, 1.0)) * sn_s) : sr * cs_s;
        sB = (float)sb;
        A = (float)(kN - sb);
        const float srf = (float)sr, crf = sqrtf(fmaxf(0.0f, __fmaf_rn(-srf, srf, 1.0f)));
        const float lam = 12.398419843320026e-7f / E32;   // mm
        Q = L.K2 * lam * lam * lam / (2.0f * srf * crf);
    } else {
        sB = 1.0f;                                        // no Bragg solution: A + sB = |k.N|
        A = (float)(kN - 1.0);
    }
    ray_rates(L, E32, Q, nb, inv_ws, sB, mu0, qr);
    if (oA && L.n_ord > 1) {
        // the other orders: sin aB_h = r_h sin aB_0, anchors in FP64 as above
        int m = nb;
        for (int h = 1; h < L.n_ord; ++h) {
            const double srh = sr * L.ord_rd[h];
            if (srh < 1.0) {
                const double sbh = sn_s != 0.0 ? __fma_rn(srh, cs_s, sqrt(__fma_rn(-srh, srh, 1.0)) * sn_s)
                                               : srh * cs_s;
                osB[h] = (float)sbh;
                oA[h] = (float)(kN - sbh);
            } else {
                osB[h] = 1.0f;
                oA[h] = (float)(kN - 1.0);
                m |= 1 << h;
            }
        }
        *nbm = m;
    }
    return true;
}

// the source polarisation projected perpendicular to k (zero if parallel)
__device__ __forceinline__ void project_pol32(const Launch32 &L, const float k[3], float p[3]) {
    const float pk = L.pol[0] * k[0] + L.pol[1] * k[1] + L.pol[2] * k[2];
    float n2 = 0.0f;
    for (int i = 0; i < 3; ++i) {
        p[i] = __fmaf_rn(-pk, k[i], L.pol[i]);
        n2 = __fmaf_rn(p[i], p[i], n2);
    }
    const float sc = n2 > 1e-12f ? rsqrtf(n2) : 0.0f;
    for (int i = 0; i < 3; ++i) p[i] *= sc;
}

// the |k.n| window of |Delta| < X* w: (sB + e1, sB + e2), clipped to [0, 1]
// (w: the rocking curve's width scale at the ray's energy)
__device__ __forceinline__ void bragg_window(const Launch32 &L, float sB, float cB, float inv_ws, float &e1,
                                             float &e2) {
    float sx = L.sx, hx2 = L.hx2;
    if (L.xs_on) {
        const float x = L.xstar / inv_ws, x2 = x * x;     // sin x and 2 sin^2(x / 2) by their series
        sx = x * __fmaf_rn(x2, __fmaf_rn(x2, 8.33333333e-3f, -0.166666667f), 1.0f);
        hx2 = 0.5f * x2 * __fmaf_rn(x2, -0.0833333333f, 1.0f);
    }
    e1 = sB <= sx ? -sB : __fmaf_rn(-sB, hx2, -cB * sx);
    e2 = cB <= sx ? 1.0f - sB : __fmaf_rn(-sB, hx2, cB * sx);
}

// acos(m / b) for b > 0 (ib = 1 / b), clamped to [0, pi], by Abramowitz & Stegun 4.4.46:
// acos(x) = sqrt(1 - x) (a0 + a1 x + ... + a7 x^7) on [0, 1] with absolute
// error <= 2e-8, acos(-x) = pi - acos(x).  1 -+ x is formed as (b -+ m) / b,
// so the result keeps its accuracy near x = +-1.  (An arc end off by 1e-6 rad
// moves the Bragg offset by b 1e-6 ~ 1e-9, far below the rocking-curve scale.)
__device__ __forceinline__ float acos_ratio(float m, float b, float ib) {
    if (m >= b) return 0.0f;
    if (m <= -b) return 3.14159265f;
    const float x = fabsf(m) * ib, omx = (b - fabsf(m)) * ib;
    float p = -0.0012624911f;
    p = __fmaf_rn(p, x, 0.0066700901f);
    p = __fmaf_rn(p, x, -0.0170881256f);
    p = __fmaf_rn(p, x, 0.0308918810f);
    p = __fmaf_rn(p, x, -0.0501743046f);
    p = __fmaf_rn(p, x, 0.0889789874f);
    p = __fmaf_rn(p, x, -0.2145988016f);
    p = __fmaf_rn(p, x, 1.5707963050f);
    const float r = sqrtf(omx) * p;
    return m >= 0.0f ? r : 3.14159265f - r;
}

// Process (b), azimuth: the arcs of xi' in [0, pi] whose cos lies in
// (iv0, iv1) / b or (iv2, iv3) / b; keep the candidate iff t3 pbar < P_xi (the
// arc measure in units of pi), then place xi' uniformly over the arcs (sign
// from the second half of the conditional uniform).  Out of line: rarely run.
// Returns (kept, cos xi', sin xi', sign).
// one arc of arc_sample: xi' in [0, pi] with cos(xi') in (lo, hi) / b, as its start
// acos(hi / b) and its length (both 0 for an empty interval)
__device__ __forceinline__ void arc_piece(float lo, float hi, float b, float ib, float &start, float &len) {
    start = 0.0f;
    len = 0.0f;
    if (lo < hi && lo < b && hi > -b) {
        start = acos_ratio(hi, b, ib);
        len = acos_ratio(lo, b, ib) - start;
    }
}

__device__ __forceinline__ float4 arc_sample(float iv0, float iv1, float iv2, float iv3, float b, float ib,
                                          float t3pbar) {
    float start[2], len[2];
    arc_piece(iv0, iv1, b, ib, start[0], len[0]);
    arc_piece(iv2, iv3, b, ib, start[1], len[1]);
    const float arcs = len[0] + len[1];
    const float pxi = arcs * 0.318309886f;
    if (!(t3pbar < pxi)) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float pos = (t3pbar / pxi) * 2.0f * arcs, sg = 1.0f;
    if (pos >= arcs) { pos -= arcs; sg = -1.0f; }
    const float xp = pos < len[0] ? start[0] + pos : start[1] + (pos - len[0]);
    float sxp, cxp;
    __sincosf(xp, &sxp, &cxp);                        // xp in [0, pi]: absolute error < 1e-6
    return make_float4(1.0f, cxp, sxp, sg);
}

// Upper bound, in units of pi, of the measure of xi' in [0, pi] with cos(xi') in
// (lo, hi) / b (ib = 1 / b), above arc_sample's FP32 value of that measure:
//   acos(c1) - acos(c2) <= (c2 - c1) / sqrt(1 - m^2), m = max(|c1|, |c2|) (acos' slope
//   is largest there; 1 - m^2 = (1 - m)(1 + m) with 1 - m = (b - |.|) / b; no bound once
//   the interval reaches +-1), and
//   acos(c1) - acos(c2) <= min(acos(c1), pi - acos(c2)) = acos(1 - e), e the smaller of
//   1 - c1 and 1 + c2 (formed as (b -+ .) / b, accurate at the edges), and
//   acos(1 - e) <= (pi / 2) sqrt(2 e) for e in [0, 2];
// 1e-4 relative and 4e-6 absolute cover FP32 rounding here and arc_sample's arccos
// (2e-8 + 2^-20 (acos + 1) per end)
__device__ __forceinline__ float arc_bound(float lo, float hi, float b, float ib) {
    if (!(lo < hi && lo < b && hi > -b)) return 0.0f;     // arc_sample's empty interval
    const float d = (hi - lo) * ib, om = (b - fmaxf(fabsf(lo), fabsf(hi))) * ib;
    const float slope = d * rsqrtf(fmaxf(om * (2.0f - om), 1e-30f));
    const float e = fminf(fminf((b - lo) * ib, (b + hi) * ib), 2.0f);
    const float edge = 2.2214415f * sqrtf(e);
    return __fmaf_rn(fminf(slope, edge), 0.318309886f * 1.0001f, 4e-6f);
}

// the tilt-grid point q_j = 2^(j/8 - 48) just below q_min (-1 below the grid); its
// table word starts process (b)
__device__ __forceinline__ int tilt_index32(float qmin) {
    if (!(qmin >= 3.5527137e-15f)) return -1;
    return min((int)floorf(8.0f * __log2f(qmin)) + 384, kQGrid - 1);
}

// Band B's arc-measure bound (units of pi) for tilts q >= q1 up to q_J on a segment
// with |k.N| in [sB + lo, sB + hi] (window |k.n| in (sB + e1, sB + e2); ca_hi =
// sqrt(1 - |k.N|max^2); is1 >= 1 / sin(theta1)): with b = c_a sin(theta), the
// window's interval of cos(xi') on the ray's side stays within |y| <= M = (D /
// sin theta1 + |k.N|max tan(theta_J / 2)) / ca_hi (D = max |S - |k.N|| from the
// small quantities), where an interval's arcsine measure is at most its width w
// over sqrt(1 - M^2); the other one lies beyond m = (S1 + |k.N|min (1 - q_J)) /
// sin theta_J (b <= sin theta_J), measure <= acos(m), 0 if m >= 1.  Margins of a
// few ulp on M, m and the result cover this function's own rounding; 1 if no
// bound applies
__device__ __forceinline__ float band_b_bound32(const Launch32 &L, float sB, float lo, float hi, float e1, float e2,
                                                float ca_hi, float is1) {
    if (!(ca_hi > 0.0f) || !(is1 > 0.0f)) return 1.0f;
    const float shi = fminf(sB + hi, 1.0f);
    const float ic = 1.0f / (ca_hi * 0.9999995f);
    const float D = fmaxf(fabsf(e1 - hi), fabsf(e2 - lo));
    const float M = __fmaf_rn(D, is1, shi * L.band_t2) * ic * 1.000001f;
    if (!(M < 1.0f)) return 1.0f;
    const float w = (e2 - e1) * is1 * ic * 1.000001f;
    float p = w * rsqrtf(__fmaf_rn(-M, M, 1.0f)) * 1.000001f;
    const float slo = fmaxf(sB + lo, 0.0f);
    const float m = __fmaf_rn(slo, 1.0f - L.band_q2, sB + e1) * L.band_is2 * 0.999999f;
    if (m < 1.0f) p += acosf(fmaxf(m, -1.0f)) * 1.000001f;
    return p * (0.318309886f * 1.000002f);
}

// Majorant of a straight segment.  Plain: mu0 + Q R_max.  Thinned: the
// scatter candidates split by their marks (v, n) into (a) v < v*, tested as
// usual; (b) v >= v*, tilt q in [q_min, 2 - q_min] and azimuth in the arcs
// where |Delta| < X*; (c) the rest, which cannot reflect and are never drawn.
// |k.N| stays in [s_lo, s_hi] on the segment (k.N is monotone along a line); a
// tilt theta < d - X*, d the distance of sin(aB + dM) from that range (never
// more than the angular distance), keeps |Delta| >= X*.  Segments with
// d <= X* keep the plain stream.  |k.N| is taken relative to sin(aB + dM)
// from the small anchors.
__device__ __forceinline__ float thin_bounds(const Launch32 &L, Lane &s, float A_exit, bool flip, bool band) {
    float la = s.qr, lb = 0.0f;
    s.ra = 1.0f;
    s.pbarB = s.pbar = 1.0f;
    s.w1 = 0u;
    if (L.irc_kind == HEART_IRC_NONE) {
        // no rocking curve: the Bragg cones' bounds (qmin, pbar: the bounds of W / W(0) on
        // the facing and the other cone; w0: the bits of the facing cone's window half-width)
        s.ra = 0.5f; s.qmin = 1.0f; s.pbar = 1.0f; s.w0 = __float_as_uint(3.14159265f);
        if (L.sampler == HEART_SAMPLER_THINNED && s.qr > 0.0f) {
            const float Ae = flip ? -2.0f * s.sB - A_exit : A_exit;
            const float lo = flip ? -s.sB : fminf(s.A, Ae), hi = fmaxf(s.A, Ae);
            const float d = lo > 0.0f ? lo : (hi < 0.0f ? -hi : 0.0f);
            const float h = 0.5f * d, h2 = h * h;
            const float sh = d < 0.1f ? h * __fmaf_rn(h2, __fmaf_rn(h2, 8.33333333e-3f, -0.166666667f), 1.0f)
                                      : __sinf(h);
            const float q0 = 2.0f * sh * sh;
            const float wn = mdf_ratio32(L, q0);
            const float wf = mdf_ratio32(L, s.sB * s.sB / (1.0f + s.cB));   // 2 sin^2(a~0 / 2)
            // the window: W <= v* W(0) where q0 + cos(a~0) cos(g_max) (1 - cos psi) >= q_v
            float psis = 3.14159265f;
            const float shi = fminf(s.sB + hi, 1.0f);
            const float cmin = s.cB * sqrtf(fmaxf(0.0f, __fmaf_rn(-shi, shi, 1.0f))) * 0.999999f;
            if (q0 < L.none_qv && cmin > 0.0f) {
                const float xq = (L.none_qv - q0) / cmin;
                if (xq < 2.0f) psis = 2.0f * asinf(sqrtf(0.5f * xq));
            }
            const float fin = wn * psis * 0.318309886f;
            const float fout = psis < 3.14159265f ? L.vstar * __fmaf_rn(-psis, 0.318309886f, 1.0f) : 0.0f;
            s.qmin = wn;
            s.pbar = wf;
            s.w0 = __float_as_uint(psis);
            la = 0.5f * s.qr * (fin + fout + wf);
        }
    } else if (L.sampler == HEART_SAMPLER_THINNED && s.qr > 0.0f) {
        // |k.N| at the exit is sB + A_exit, or -(sB + A_exit) if k.N changed sign
        const float Ae = flip ? -2.0f * s.sB - A_exit : A_exit;
        const float lo = flip ? -s.sB : fminf(s.A, Ae);   // relative to sB; |k.N| passes 0 on a flip
        const float hi = fmaxf(s.A, Ae);
        const float d = lo > 0.0f ? lo : (hi < 0.0f ? -hi : 0.0f);
        float tmin = d - (L.xs_on ? L.xstar / s.inv_ws : L.xstar);
        if (tmin > 0.0f) {
            tmin = fminf(tmin, 1.57079637f);
            // sin to float precision: a short series below 0.1 rad, the SFU above (far off Bragg)
            const float h = 0.5f * tmin, h2 = h * h;
            const float sh = tmin < 0.1f ? h * __fmaf_rn(h2, __fmaf_rn(h2, 8.33333333e-3f, -0.166666667f), 1.0f)
                                         : __sinf(h);
            const float st = 2.0f * sh * sqrtf(fmaxf(0.0f, __fmaf_rn(-sh, sh, 1.0f)));   // sin(theta_min)
            s.qmin = 2.0f * sh * sh;
            const int j0 = tilt_index32(s.qmin);
            s.w0 = j0 < 0 ? 0u : L.qgrid[j0];
            // arc bound: two |k.n| windows of width S2 - S1 over b >= cos(a_hi) sin(theta_min)
            const float shi = fminf(s.sB + hi, 1.0f);
            const float ca_hi = sqrtf(fmaxf(0.0f, __fmaf_rn(-shi, shi, 1.0f)));
            const float bmin = ca_hi * st * 0.999999f;
            float e1, e2;
            bragg_window(L, s.sB, s.cB, s.inv_ws, e1, e2);
            // two windows of width w in cos(xi'), each of arc measure <= acos(1 - w) / pi
            const float w = (e2 - e1) / bmin;
            if (w >= 2.0f || !(bmin > 0.0f)) {
                s.pbar = 1.0f;
            } else if (w <= 0.18f) {
                // acos(1 - w) = 2 asin(t), t = sqrt(w / 2) <= 0.3: asin by its Taylor series to t^9
                // (all terms positive; the rest is below 2e-7 relative, inside the 1e-6 margin)
                const float t2 = 0.5f * w, t = sqrtf(t2);
                float p = __fmaf_rn(t2, 0.0303819444f, 0.0446428571f);
                p = __fmaf_rn(p, t2, 0.075f);
                p = __fmaf_rn(p, t2, 0.166666667f);
                p = __fmaf_rn(p, t2, 1.0f);
                s.pbar = fminf(1.0f, 1.27323954f * t * p * 1.000001f);
            } else {
                s.pbar = fminf(1.0f, 0.636619772f * acosf(1.0f - w) * 1.000001f);
            }
            // band B (one order): from the grid point kBandDJ steps above q_min's, its
            // tilts from the table knot that starts its first word's interval
            s.w1 = s.w0;
            s.pbarB = s.pbar;
            float pw = (float)((1ull << 32) - s.w0) * 2.3283064365386963e-10f * s.pbar;
            if (band && j0 >= 0 && j0 + kBandDJ < kBandJ2) {
                const uint32_t w1 = L.qgrid[j0 + kBandDJ];
                if (w1 < L.band_w2) {
                    const float pB = band_b_bound32(L, s.sB, lo, hi, e1, e2, ca_hi, L.band_is1[j0 + kBandDJ]);
                    if (pB < s.pbar) {
                        s.w1 = w1;
                        s.pbarB = pB;
                        const float fA = (float)((w1 - s.w0) + (0u - L.band_w2)) * s.pbar;
                        const float fB = (float)(L.band_w2 - w1) * pB;
                        pw = (fA + fB) * 2.3283064365386963e-10f;
                    }
                }
            }
            la = s.qr * L.vstar;
            lb = s.qr * (1.0f - L.vstar) * pw;
            s.ra = la / (la + lb);
        }
    }
    return la + lb;
}

// the segment's majorant mu0 + lam: 1 / mu, the absorption share and its word threshold
__device__ __forceinline__ void set_majorant(Lane &s, float lam) {
    const float mu = s.mu0 + lam;
    s.inv_mu = 1.0f / mu;
    s.pa = s.mu0 / mu;
    s.inv_1mpa = s.pa < 1.0f ? 1.0f / (1.0f - s.pa) : 0.0f;
    // absorb iff (w + 1/2) 2^-32 < pa  <=>  w < ceil(pa 2^32 - 1/2)
    s.pa_thr = s.pa >= 1.0f ? 0xFFFFFFFFu : __float2uint_ru(fminf(s.pa * 4294967296.0f, 4294967040.0f));
}

__device__ __forceinline__ void thin_segment(const Launch32 &L, Lane &s, float A_exit, bool flip) {
    set_majorant(s, thin_bounds(L, s, A_exit, flip, L.n_ord == 1));
}

// Several reflection orders (Sec. 2.2.3: the rate sums over H): every order's
// anchor moved with the current order's (a reflection, or the walk along a
// cylinder, changes |k.N| alike for all), each order's bounds on the segment
// (dex: the change of the anchors to the exit), the cumulative shares of the
// candidate rate and the majorant mu0 + sum of the orders' rates.
__device__ __forceinline__ void thin_orders(const Launch32 &L, Lane &s, float dex, bool flip) {
    const float dA = s.A - s.oA[s.h];
    float lam = 0.0f;
    for (int g = 0; g < L.n_ord; ++g) {
        const float Ag = g == s.h ? s.A : s.oA[g] + dA;
        s.oA[g] = Ag;
        s.A = Ag;
        s.sB = s.osB[g];
        s.cB = s.ocB[g];
        s.qr = s.oqr[g];
        s.inv_ws = s.oiw[g];
        lam += thin_bounds(L, s, Ag + dex, flip, false);      // several orders: no band B
        s.ora[g] = s.ra;
        s.oqmin[g] = s.qmin;
        s.opbar[g] = s.pbar;
        s.ow0[g] = s.w0;
        s.ocum[g] = lam;
    }
    for (int g = 0; g < L.n_ord; ++g) s.ocum[g] = lam > 0.0f ? s.ocum[g] / lam : 1.0f;
    s.ocum[L.n_ord - 1] = 1.0f;
    s.h = L.n_ord - 1;                                        // the fields hold the last order's values
    set_majorant(s, lam);
}

// the current candidate's order (the extended kernel with several orders)
__device__ __forceinline__ void load_order(Lane &s, int h) {
    s.h = h;
    s.A = s.oA[h];
    s.sB = s.osB[h];
    s.cB = s.ocB[h];
    s.qr = s.oqr[h];
    s.inv_ws = s.oiw[h];
    s.ra = s.ora[h];
    s.qmin = s.oqmin[h];
    s.pbar = s.opbar[h];
    s.pbarB = s.pbar;                                     // several orders: no band B
    s.w0 = s.ow0[h];
}

// A ray with several orders as a lane takes it: every order's anchor and sine
// (oa, os), cosine, inverse width scale and rate at the ray's energy (sin aB_h
// = r_h sin aB_0 only sets Q_h here, so FP32 rounding of E is harmless); nbm
// marks the orders without a Bragg solution.  The fields hold order 0.
__device__ __forceinline__ void start_orders(const Launch32 &L, Lane &s, const float oa[HEART_MAX_ORDERS],
                                             const float os[HEART_MAX_ORDERS], int nbm) {
    float ws = 1.0f, sh = 0.0f;
    if (L.n_irc_e > 0) irc_energy32(L, s.E, ws, sh);
    const float iws = 1.0f / ws;
    const float lam = 12.398419843320026e-7f / s.E;         // mm
    const float s1 = (float)L.hc_2d / s.E;                  // sin aB of order 0
    float mu0;
    for (int h = 0; h < L.n_ord; ++h) {
        const int nb = (nbm >> h) & 1;
        s.oA[h] = oa[h];
        s.osB[h] = os[h];
        s.ocB[h] = sqrtf(fmaxf(0.0f, __fmaf_rn(-os[h], os[h], 1.0f)));
        s.oiw[h] = L.ord_iw[h] * iws;
        float Q = 0.0f;
        if (!nb) {
            const float sr = fminf(s1 * L.ord_r[h], 1.0f);
            const float cr = sqrtf(fmaxf(0.0f, __fmaf_rn(-sr, sr, 1.0f)));
            Q = cr > 0.0f ? L.ord_k2[h] * lam * lam * lam / (2.0f * sr * cr) : 0.0f;
        }
        ray_rates(L, s.E, Q, nb, s.oiw[h], os[h], mu0, s.oqr[h]);
    }
    s.no_bragg = nbm == (1 << L.n_ord) - 1;
    s.h = 0;
    s.A = s.oA[0];
    s.sB = s.osB[0];
    s.cB = s.ocB[0];
    s.qr = s.oqr[0];
    s.inv_ws = s.oiw[0];
}

// start a straight segment at x0 along k; s.A, s.sgn, s.sB and (cylinder) s.rho0 are set
// cylinder: constants of k.N along the segment from x0: r(l)^2 = r0^2 (1 + l (cb1 + l cb2))
template <int GEOM_T>
__device__ __forceinline__ void segment_consts(const Launch32 &L, Lane &s) {
    const int GEOM = GEOM_T >= 0 ? GEOM_T : L.geometry;
    s.Lsum = 0.0f;
    s.Lcomp = 0.0f;
    if (GEOM != HEART_FLAT) {
        const float r0 = L.R + s.rho0;
        const float X = s.x0[1], Y = s.x0[2];
        const float kappa = s.sgn * (s.sB + s.A);           // k.N at x0
        const float aa = __fmaf_rn(s.k[1], s.k[1], s.k[2] * s.k[2]);
        const float bb = -kappa * r0;                        // (X, Y) . (kX, kY)
        const float ir0 = 1.0f / r0;
        s.cb1 = 2.0f * bb * ir0 * ir0;
        s.cb2 = aa * ir0 * ir0;
        s.cga = aa * ir0;
        s.ck0 = kappa;
        s.ctau0 = (X * s.k[2] - Y * s.k[1]) * ir0;          // k . t2 at x0 (t2 = N x axis)
    }
}

template <int GEOM_T, bool ORD = false>
__device__ __forceinline__ void segment(const Launch32 &L, Lane &s) {
    const int GEOM = GEOM_T >= 0 ? GEOM_T : L.geometry;
    segment_consts<GEOM_T>(L, s);
    float best = 3.0e38f;
    int face = HEART_EXIT_SIDE;
    auto cand = [&](float v, int f) {
        v = fmaxf(v, 0.0f);
        if (v < best) { best = v; face = f; }
    };
    if (GEOM == HEART_FLAT) {
        const float h = s.x0[2], a = s.x0[0], b = s.x0[1];
        const float kh = s.k[2], ka = s.k[0], kb = s.k[1];
        if (kh > 0) cand(-h / kh, HEART_EXIT_FRONT);
        if (kh < 0) cand((-L.thick - h) / kh, HEART_EXIT_BACK);
        if (ka > 0) cand((L.half_d - a) / ka, HEART_EXIT_SIDE);
        if (ka < 0) cand((-L.half_d - a) / ka, HEART_EXIT_SIDE);
        if (kb > 0) cand((L.half_n - b) / kb, HEART_EXIT_SIDE);
        if (kb < 0) cand((-L.half_n - b) / kb, HEART_EXIT_SIDE);
    } else {
        const float R = L.R, t = L.thick, rho = s.rho0;
        const float r0 = R + rho;
        const float X = s.x0[1], Y = s.x0[2];
        const float kappa = s.sgn * (s.sB + s.A);           // k.N at x0
        const float aa = __fmaf_rn(s.k[1], s.k[1], s.k[2] * s.k[2]);
        const float bb = -kappa * r0;                        // (X, Y) . (kX, kY)
        const float ci = rho * (2.0f * R + rho);             // r^2 - R^2
        const float co = (rho - t) * (2.0f * R + rho + t);   // r^2 - (R + t)^2
        if (aa > 0.0f) {
            if (bb < 0.0f) {
                const float disc = __fmaf_rn(bb, bb, -aa * ci);
                if (disc >= 0.0f) cand(ci / (sqrtf(disc) - bb), HEART_EXIT_FRONT);
            }
            const float sq = sqrtf(fmaxf(__fmaf_rn(bb, bb, -aa * co), 0.0f));
            cand(bb > 0.0f ? -co / (bb + sq) : (sq - bb) / aa, HEART_EXIT_BACK);
        }
        const float z = s.x0[0] - L.zc, kz = s.k[0];
        if (kz > 0) cand((L.half_d - z) / kz, HEART_EXIT_SIDE);
        if (kz < 0) cand((-L.half_d - z) / kz, HEART_EXIT_SIDE);
        const float gp = -X * L.sphi + Y * L.cphi, rp = -s.k[1] * L.sphi + s.k[2] * L.cphi;
        if (rp > 0) cand(-gp / rp, HEART_EXIT_SIDE);
        const float gm = -X * L.sphi - Y * L.cphi, rm = -s.k[1] * L.sphi - s.k[2] * L.cphi;
        if (rm > 0) cand(-gm / rm, HEART_EXIT_SIDE);
    }
    s.s_exit = best;
    s.face = face;
    // anchor at the exit point (cylinder: k.N changes along the segment)
    float A_exit = s.A;
    bool flip = false;
    if (GEOM != HEART_FLAT) {
        const float Lp = fminf(best, 1.0e6f);
        const float eps = Lp * __fmaf_rn(Lp, s.cb2, s.cb1);
        const float rho = sqrtf(fmaxf(1.0f + eps, 1e-30f));
        const float dk = (s.ck0 * (-eps / (1.0f + rho)) - Lp * s.cga) / rho;
        A_exit = __fmaf_rn(s.sgn, dk, s.A);
        flip = s.sB + A_exit < 0.0f;
    }
    if (ORD && L.n_ord > 1) thin_orders(L, s, A_exit - s.A, flip);
    else thin_segment(L, s, A_exit, flip);
}

__device__ __forceinline__ void to_global(const Launch32 &L, const float *p, double *g, bool point) {
    for (int i = 0; i < 3; ++i)
        g[i] = (point ? L.fc[i] : 0.0) + (double)p[0] * L.fa[0][i] + (double)p[1] * L.fa[1][i] +
               (double)p[2] * L.fa[2][i];
}

__device__ __forceinline__ float qe32(const Launch32 &L, float E) {
    if (L.n_qe <= 0) return 1.0f;
    if (E <= L.qe_e[0]) return L.qe_v[0];
    for (int i = 1; i < L.n_qe; ++i)
        if (E <= L.qe_e[i]) {
            const float f = (E - L.qe_e[i - 1]) / (L.qe_e[i] - L.qe_e[i - 1]);
            return __fmaf_rn(f, L.qe_v[i] - L.qe_v[i - 1], L.qe_v[i - 1]);
        }
    return L.qe_v[L.n_qe - 1];
}

// tally slots in shared memory (32-bit per chunk, flushed as 64-bit)
struct BlockTally {
    unsigned int t[kTallyN];
    unsigned long long coll, emit, miss;
};

// a ray's record (tests): written out of line, so that kernels that may write
// records keep the registers of those that never do
__device__ __forceinline__ void write_record(const Launch32 &L, const Lane &s, int outcome, float xe0, float xe1,
                                          float xe2, float u, float v, int ix, int iy, int hit, bool pol) {
    const uint64_t ray = ((uint64_t)s.rh << 32) | s.rl;
    heart_ray_record &o = L.rec[ray - L.offset];
    const float xe[3] = {xe0, xe1, xe2};
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
    if (pol) to_global(L, s.p, o.pol, false);
    else o.pol[0] = o.pol[1] = o.pol[2] = 0.0;
}

// the record of a ray that did not enter, or entered with an invalid energy (a miss)
__device__ __forceinline__ void write_miss_record(const Launch32 &L, uint64_t ray, const float x[3], const float k[3],
                                               float E, const float p[3]) {
    heart_ray_record &o = L.rec[ray - L.offset];
    o.ray_id = ray;
    o.outcome = HEART_MISS;
    o.nrefl = 0;
    o.ncoll = 0;
    o.energy_keV = E;
    to_global(L, x, o.pos, true);
    to_global(L, k, o.dir, false);
    o.u_mm = __longlong_as_double(0x7ff8000000000000LL);
    o.v_mm = o.u_mm;
    o.ix = -1;
    o.iy = -1;
    o.det_hit = 0;
    o.no_bragg = 0;
    to_global(L, p, o.pol, false);
}

// finish a ray: detector projection + binning + tallies (+ record when REC and
// the launch asks for records)
template <bool REC, bool EXT>
__device__ __forceinline__ void finish(const Launch32 &L, Lane &s, int outcome, BlockTally &bt) {
    int ix = -1, iy = -1, hit = 0;
    float u = __int_as_float(0x7fc00000), v = u;
    const bool out = outcome == HEART_EXIT_FRONT || outcome == HEART_EXIT_BACK || outcome == HEART_EXIT_SIDE;
    const float len = out ? s.s_exit : s.Lsum;
    float xe[3];
    for (int i = 0; i < 3; ++i) xe[i] = __fmaf_rn(len, s.k[i], s.x0[i]);
    if (out) {
        const float rel[3] = {L.D0[0] - xe[0], L.D0[1] - xe[1], L.D0[2] - xe[2]};
        const float den = s.k[0] * L.nd[0] + s.k[1] * L.nd[1] + s.k[2] * L.nd[2];
        if (den != 0.0f) {
            const float t = (rel[0] * L.nd[0] + rel[1] * L.nd[1] + rel[2] * L.nd[2]) / den;
            if (t > 0.0f) {
                const float P[3] = {__fmaf_rn(t, s.k[0], -rel[0]), __fmaf_rn(t, s.k[1], -rel[1]),
                                    __fmaf_rn(t, s.k[2], -rel[2])};
                u = P[0] * L.eu[0] + P[1] * L.eu[1] + P[2] * L.eu[2];
                v = P[0] * L.ev[0] + P[1] * L.ev[1] + P[2] * L.ev[2];
                const float fx = __fmaf_rn(u, L.inv_pix, L.hnx), fy = __fmaf_rn(v, L.inv_pix, L.hny);
                if (fx >= 0.0f && fx < (float)L.nx && fy >= 0.0f && fy < (float)L.ny) {
                    ix = min((int)fx, L.nx - 1);
                    iy = min((int)fy, L.ny - 1);
                    hit = 1;
                    const size_t idx = (size_t)iy * (size_t)L.nx + (size_t)ix;
                    if (L.count64) atomicAdd((unsigned long long *)L.img + idx, 1ull);
                    else atomicAdd((int *)L.img + idx, 1);
                    atomicAdd(&bt.t[T_DET_HITS], 1u);
                    if (L.eimg)
                        atomicAdd(L.eimg + idx, (unsigned long long)__float2ll_rn(s.E * qe32(L, s.E) * 1.0e6f));
                }
            }
        }
    }
    atomicAdd(&bt.t[T_ABSORBED + (outcome - HEART_ABSORBED)], 1u);
    atomicAdd(&bt.t[T_HIST0 + (s.nrefl < 15 ? s.nrefl : 15)], 1u);
    if (s.no_bragg) atomicAdd(&bt.t[T_NO_BRAGG], 1u);
    if (REC && L.rec) write_record(L, s, outcome, xe[0], xe[1], xe[2], u, v, ix, iy, hit, EXT && s.pol);
}

// one tentative collision; returns an outcome code, or -1 while the ray lives
// crystallite normal n at the current collision in the crystal frame, and on
// a cylinder the radial change drho of the collision point from the segment start
template <int GEOM_T>
__device__ __forceinline__ void crystallite_normal(const Launch32 &L, const Lane &s, float st, float sx, float cx,
                                                   float q, float eps, float rho, float n[3], float &drho) {
    const int GEOM = GEOM_T >= 0 ? GEOM_T : L.geometry;
    const float ct = 1.0f - q;
    if (GEOM == HEART_FLAT) {
        n[0] = st * cx; n[1] = st * sx; n[2] = ct;
        drho = 0.0f;
    } else {
        const float X = __fmaf_rn(s.Lsum, s.k[1], s.x0[1]), Y = __fmaf_rn(s.Lsum, s.k[2], s.x0[2]);
        drho = (L.R + s.rho0) * eps / (1.0f + rho);           // r - r0 at the collision
        const float ir = 1.0f / (L.R + s.rho0 + drho);
        const float sxs = st * sx;
        n[0] = st * cx;
        n[1] = (-ct * X - sxs * Y) * ir;
        n[2] = (-ct * Y + sxs * X) * ir;
    }
}

// A scatter candidate without rocking curve (R a delta function): the
// crystallite normal on the Bragg cone k.n = sg sin(a~0), a~0 = aB + Delta_M,
// at azimuth psi about k measured from the part of N perpendicular to k.
// Plain: sg = +1 if the top bit of u2 is set, psi = 2 pi u3, kept with
// probability W(q) G / W(0).  Thinned: u2 picks the facing cone's window
// |psi| < psis (bound W at the segment's smallest tilt), the rest of the facing
// cone (bound v* W(0)) or the other cone, psi uniform over the part, kept with
// probability W(q) G / (the part's bound).  In the collision's frame (t1, t2, N) with k = (k0, kt, kN)
// and c = sqrt(1 - kN^2): e1 = (-kN k0, -kN kt, c^2) / c, e2 = (kt, -k0, 0) / c,
// and the tilt q = 1 - n.N = q0 + c0 c (1 - cos psi) with q0 = 1 - cos(g -+ a~0),
// sin g = |kN|.  On the cone facing the ray (sg = sign kN) q0 comes from the
// anchor Ac = |kN| - sin a~0 without cancellation:
//   q0 = Ac^2 (c0 + s0 (2 s0 + Ac) / (c0 + c)) / (c0 + c).
template <int GEOM_T, bool EXT, bool ORD>
__device__ __forceinline__ int cone_step(const Launch32 &L, Lane &s, uint32_t w2, uint32_t w3, float v, float Ac,
                                         float kN, float kt2, float eps, float rho) {
    const int GEOM = GEOM_T >= 0 ? GEOM_T : L.geometry;
    const float s0 = s.sB, c0 = s.cB;
    const float sa = s0 + Ac;                                   // |k.N| at the collision
    const float cb = sqrtf(fmaxf(0.0f, __fmaf_rn(-sa, sa, 1.0f)));
    // the cone: thinned, the facing cone's window |psi| < psis, the rest of the facing cone
    // (k.n of the sign of k.N) or the other cone by their shares of the segment's bound
    // (lane fields qmin, pbar: W / W(0) bounds; w0: psis); plain, the cone by the top bit.
    // psi / (2 pi) = x0 + xs u3
    float sg, wb = 1.0f, x0 = 0.0f, xs = 1.0f;
    if (L.sampler == HEART_SAMPLER_THINNED) {
        const float psis = __uint_as_float(s.w0);
        const float fin = s.qmin * psis * 0.318309886f;
        const float fout = psis < 3.14159265f ? L.vstar * __fmaf_rn(-psis, 0.318309886f, 1.0f) : 0.0f;
        const float t2 = u01_32(w2) * (fin + fout + s.pbar);
        const float hw = psis * 0.159154943f;                  // psis / (2 pi)
        if (t2 < fin) { sg = s.sgn; wb = s.qmin; x0 = -hw; xs = 2.0f * hw; }
        else if (t2 < fin + fout) { sg = s.sgn; wb = L.vstar; x0 = hw; xs = 1.0f - 2.0f * hw; }
        else { sg = -s.sgn; wb = s.pbar; }
    } else {
        sg = (w2 & 0x80000000u) ? 1.0f : -1.0f;
    }
    float q0;
    if (sg == s.sgn) {
        const float cs = c0 + cb;
        q0 = Ac * Ac * __fdividef(__fmaf_rn(s0, __fdividef(__fmaf_rn(2.0f, s0, Ac), cs), c0), cs);
    } else {
        q0 = __fmaf_rn(s0, sa, __fmaf_rn(-c0, cb, 1.0f));       // 1 - cos(g + a~0)
    }
    float sh, ch;
    sincospif(__fmaf_rn(xs, u01_32(w3), x0), &sh, &ch);      // psi / 2, accurate near 0
    const float C = c0 * cb;
    const float omc = 2.0f * sh * sh;                           // 1 - cos psi
    const float q = __fmaf_rn(C, omc, q0);
    // n in the collision frame
    const float k0 = s.k[0], cp = 1.0f - omc, sp = 2.0f * sh * ch;
    const float ic = cb > 1e-20f ? 1.0f / cb : 0.0f;
    float nl0, nl1;
    if (cb > 1e-20f) {
        nl0 = __fmaf_rn(sg * s0, k0, c0 * (__fmaf_rn(cp, -kN * k0, sp * kt2)) * ic);
        nl1 = __fmaf_rn(sg * s0, kt2, c0 * (__fmaf_rn(cp, -kN * kt2, -sp * k0)) * ic);
    } else {                                                    // k along N: any axes perpendicular to k
        nl0 = c0 * cp;
        nl1 = c0 * sp;
    }
    float n[3], drho = 0.0f, G;
    crystallite_normal<GEOM_T>(L, s, 1.0f, nl1, nl0, q, eps, rho, n, drho);
    const float kn = sg * s0;                                   // k.n
    if (EXT && s.pol) {
        float pk = 0.0f, pn = 0.0f;
        for (int i = 0; i < 3; ++i) { pk = __fmaf_rn(s.p[i], s.k[i], pk); pn = __fmaf_rn(s.p[i], n[i], pn); }
        const float pks = __fmaf_rn(-2.0f * kn, pn, pk);
        G = __fmaf_rn(-pks, pks, 1.0f);                         // Eq. (G_pol)
    } else {
        const float c2 = __fmaf_rn(-2.0f * s0, s0, 1.0f);
        G = 0.5f * __fmaf_rn(c2, c2, 1.0f);                     // Eq. (G_unpol) at a~0
    }
    if (!(v * wb < mdf_ratio32(L, q) * G)) return -1;
    ++s.nrefl;
    if (s.nrefl > L.max_refl) return HEART_CAPPED;
    if (GEOM != HEART_FLAT) s.rho0 += drho;
    float kk = 0.0f;
    for (int i = 0; i < 3; ++i) {
        s.x0[i] = __fmaf_rn(s.Lsum, s.k[i], s.x0[i]);
        s.k[i] = __fmaf_rn(-2.0f * kn, n[i], s.k[i]);
        kk = __fmaf_rn(s.k[i], s.k[i], kk);
    }
    const float sc = rsqrtf(kk);
    for (int i = 0; i < 3; ++i) s.k[i] *= sc;
    if (EXT && s.pol) {
        float pk = 0.0f;
        for (int i = 0; i < 3; ++i) pk = __fmaf_rn(s.p[i], s.k[i], pk);
        float pp = 0.0f;
        for (int i = 0; i < 3; ++i) { s.p[i] = __fmaf_rn(-pk, s.k[i], s.p[i]); pp = __fmaf_rn(s.p[i], s.p[i], pp); }
        const float ps = rsqrtf(pp);
        for (int i = 0; i < 3; ++i) s.p[i] *= ps;
    }
    // k'.N = sign(kN) T: T = Ac - s0 + 2 q s0 on the facing cone, sa + 2 s0 (1 - q) on the other
    const float T = (sg == s.sgn) ? __fmaf_rn(2.0f * q, s0, Ac - s0) : __fmaf_rn(2.0f * s0, 1.0f - q, sa);
    if (T < 0.0f) {
        s.A = (sg == s.sgn) ? __fmaf_rn(-2.0f * q, s0, -Ac) : -T - s0;
        s.sgn = -s.sgn;
    } else {
        s.A = T - s0;
    }
    segment<GEOM_T, ORD>(L, s);
    return -1;
}

// ORD (the persistent extended kernel only): several reflection orders
template <int GEOM_T, int IRC, bool EXT, bool ORD = false>
__device__ __forceinline__ int step(const Launch32 &L, Lane &s, const float *tab) {
    const int GEOM = GEOM_T >= 0 ? GEOM_T : L.geometry;
    if (s.ncoll >= L.max_coll) return HEART_STUCK;
    uint32_t w[4];
    philox_l<(GEOM_T >= 0)>(L, s.rl, s.rh, s.call++, 0u, w);
    const float l = -__logf(u01_32(w[0])) * s.inv_mu;
    // Kahan-compensated path length along the segment
    const float y = l - s.Lcomp;
    const float t = s.Lsum + y;
    s.Lcomp = (t - s.Lsum) - y;
    if (t > s.s_exit) return s.face;
    s.Lsum = t;
    ++s.ncoll;
    if (w[1] < s.pa_thr) return HEART_ABSORBED;
    float v = (u01_32(w[1]) - s.pa) * s.inv_1mpa;
    if (ORD && L.n_ord > 1) {
        // the reflection order by its share of the candidate rate (sum over H); the
        // conditional uniform stays the acceptance uniform
        int h = 0;
        while (h < L.n_ord - 1 && !(v < s.ocum[h])) ++h;
        const float c0 = h > 0 ? s.ocum[h - 1] : 0.0f;
        v = (v - c0) / (s.ocum[h] - c0);
        load_order(s, h);
    }
    // k.t2 and k.N at the collision point (cylinder: from the along-segment length)
    float dk = 0.0f, eps = 0.0f, rho = 1.0f, kt2, kN;
    if (GEOM == HEART_FLAT) {
        kt2 = s.k[1];
        kN = s.k[2];
    } else {
        const float Lp = s.Lsum;
        eps = Lp * __fmaf_rn(Lp, s.cb2, s.cb1);
        rho = sqrtf(1.0f + eps);
        const float rinv = 1.0f / rho;
        dk = (s.ck0 * (-eps / (1.0f + rho)) - Lp * s.cga) * rinv;
        kt2 = s.ctau0 * rinv;
        kN = s.ck0 + dk;
    }
    const float Ac = __fmaf_rn(s.sgn, dk, s.A);               // anchor at the collision point
    if ((IRC >= 0 ? IRC : L.irc_kind) == HEART_IRC_NONE) return cone_step<GEOM_T, EXT, ORD>(L, s, w[2], w[3], v, Ac, kN, kt2, eps, rho);
    // the candidate's stream: (a), or the plain stream, takes the table word over
    // its full range, (b) maps it onto [w0, 2^32); one table lookup for both
    // (a warp almost always holds candidates of both streams)
    const bool in_a = v < s.ra;
    uint32_t wq = w[2];
    float pb = s.pbar;                                        // (b): the candidate's band's arc bound
    if (in_a) {
        v = s.ra < 1.0f ? (v / s.ra) * L.vstar : v;
    } else {
        float vb = (v - s.ra) / (1.0f - s.ra);
        if (s.pbarB < s.pbar) {
            // two bands: A, words [w0, w1) and [w2, 2^32) at pbar, by its share of the rate;
            // B, words [w1, w2) at pbarB
            const uint32_t spanA = (s.w1 - s.w0) + (0u - L.band_w2), spanB = L.band_w2 - s.w1;
            const float fA = (float)spanA * s.pbar, fB = (float)spanB * s.pbarB;
            const float t = vb * (fA + fB);
            if (t < fA) {
                vb = t / fA;
                wq = s.w0 + __umulhi(w[2], spanA);
                if (wq >= s.w1) wq += spanB;
            } else {
                vb = (t - fA) / fB;
                wq = s.w1 + __umulhi(w[2], spanB);
                pb = s.pbarB;
            }
        } else {
            wq = s.w0 + __umulhi(w[2], 0u - s.w0) + (s.w0 == 0u ? w[2] : 0u);
        }
        v = __fmaf_rn(1.0f - L.vstar, vb, L.vstar);
    }
    const float q = mdf_q32(tab, wq);
    if (!in_a && (q < s.qmin || q > 2.0f - s.qmin)) return -1;   // (b): cannot reflect
    const float st = sqrtf(q * (2.0f - q));
    float sx, cx, D;
    if (in_a) {                                               // process (a), or the plain stream
        sincos_2pi(u01_32(w[3]), &sx, &cx);
        D = __fmaf_rn(st, __fmaf_rn(s.k[0], cx, kt2 * sx), -q * kN);
    } else {                                                  // process (b)
        const float ca = sqrtf(__fmaf_rn(s.k[0], s.k[0], kt2 * kt2));
        const float b = ca * st, ib = 1.0f / b;
        // intervals of y = cos(xi - xi_k) with |k.n| = |kN (1 - q) + b y| in the window,
        // the same-side one from small quantities
        float e1, e2;
        bragg_window(L, s.sB, s.cB, s.inv_ws, e1, e2);
        const float sa = s.sB + Ac;                           // |k.N| here while k.N keeps its sign
        // interval ends times b: (iv[0], iv[1]) then (iv[2], iv[3])
        float iv[4];
        if (sa > 0.0f) {
            const float m1 = __fmaf_rn(sa, q, e1 - Ac), m2 = __fmaf_rn(sa, q, e2 - Ac);
            const float p1 = __fmaf_rn(sa, 1.0f - q, s.sB + e1), p2 = __fmaf_rn(sa, 1.0f - q, s.sB + e2);
            if (s.sgn > 0.0f) { iv[0] = m1; iv[1] = m2; iv[2] = -p2; iv[3] = -p1; }
            else { iv[0] = p1; iv[1] = p2; iv[2] = -m2; iv[3] = -m1; }
        } else {
            const float a = kN * (1.0f - q), S1 = s.sB + e1, S2 = s.sB + e2;
            iv[0] = S1 - a; iv[1] = S2 - a; iv[2] = -S2 - a; iv[3] = -S1 - a;
        }
        const float t3pbar = u01_32(w[3]) * pb;
        // P_xi <= 2 acos(1 - w) / pi <= sqrt(2 w), w = (S2 - S1) / b: half of the candidates end here
        if (t3pbar * t3pbar * b >= 2.0002f * (e2 - e1)) return -1;
        // a tighter bound before the arcs themselves (most of the rest end here); it lies
        // above arc_sample's measure, so no candidate that arc_sample keeps ends here
        if (t3pbar >= arc_bound(iv[0], iv[1], b, ib) + arc_bound(iv[2], iv[3], b, ib)) return -1;
        const float4 r = arc_sample(iv[0], iv[1], iv[2], iv[3], b, ib, t3pbar);
        if (r.x == 0.0f) return -1;                           // outside the arcs: cannot reflect
        const float cxp = r.y, sxp = r.z, sg = r.w;
        const float ica = ib * st;                            // 1 / ca
        cx = (s.k[0] * cxp - sg * kt2 * sxp) * ica;           // xi = xi_k + sg xp
        sx = (kt2 * cxp + sg * s.k[0] * sxp) * ica;
        D = __fmaf_rn(st * ca, cxp, -q * kN);
    }
    const float e = __fmaf_rn(s.sgn, D, Ac);                  // |k.n| - sin(aB + Delta_M)
    if (v >= irc_bound32<IRC>(L, fabsf(e) * s.inv_ws)) return -1;   // rejected whatever Delta is
    float sa = s.sB + e;
    float delta;
    if (sa > 0.0f) {
        sa = fminf(sa, 1.0f);
        const float cs = sqrtf(fmaxf(0.0f, 1.0f - sa * sa));
        const float t = fmaxf(-1.0f, fminf(1.0f, e * (2.0f * s.sB + e) / __fmaf_rn(sa, s.cB, s.sB * cs)));
        // asin t = t + t^3/6 + 3 t^5/40 + ... : three terms reach FP32 rounding for |t| < 0.01
        const float t2 = t * t;
        delta = fabsf(t) < 0.01f ? __fmaf_rn(t * t2, __fmaf_rn(t2, 0.075f, 0.166666667f), t) : asinf(t);
    } else {
        sa = fminf(-sa, 1.0f);                                 // the normal flipped side
        delta = asinf(sa) - asinf(s.sB);
    }
    const float kn = s.sgn * (s.sB + e);                       // k.n
    float n[3], drho = 0.0f, G;
    bool have_n = false;
    if (EXT && s.pol) {
        // Eq. (G_pol): G = 1 - (p . k_s)^2, k_s = k - 2 (k.n) n
        crystallite_normal<GEOM_T>(L, s, st, sx, cx, q, eps, rho, n, drho);
        have_n = true;
        float pk = 0.0f, pn = 0.0f;
        for (int i = 0; i < 3; ++i) { pk = __fmaf_rn(s.p[i], s.k[i], pk); pn = __fmaf_rn(s.p[i], n[i], pn); }
        const float pks = __fmaf_rn(-2.0f * kn, pn, pk);
        G = __fmaf_rn(-pks, pks, 1.0f);
    } else {
        const float c2 = __fmaf_rn(-2.0f * sa, sa, 1.0f);
        G = 0.5f * __fmaf_rn(c2, c2, 1.0f);                    // Eq. (G_unpol)
    }
    if (v < irc_rel32<IRC>(L, delta * s.inv_ws) * G) {    // R(x / w) / R_max
        ++s.nrefl;
        if (s.nrefl > L.max_refl) return HEART_CAPPED;
        // reflection k <- k - 2 (k.n) n (Sec. 2.2.4)
        if (!have_n) crystallite_normal<GEOM_T>(L, s, st, sx, cx, q, eps, rho, n, drho);
        if (GEOM != HEART_FLAT) s.rho0 += drho;                // depth of the new segment start
        float kk = 0.0f;
        for (int i = 0; i < 3; ++i) {
            s.x0[i] = __fmaf_rn(s.Lsum, s.k[i], s.x0[i]);
            s.k[i] = __fmaf_rn(-2.0f * kn, n[i], s.k[i]);
            kk = __fmaf_rn(s.k[i], s.k[i], kk);
        }
        const float sc = rsqrtf(kk);
        for (int i = 0; i < 3; ++i) s.k[i] *= sc;
        if (EXT && s.pol) {
            // p_s = (p - (p.k_s) k_s) / |...| (Sec. 2.2.4)
            float pk = 0.0f;
            for (int i = 0; i < 3; ++i) pk = __fmaf_rn(s.p[i], s.k[i], pk);
            float pp = 0.0f;
            for (int i = 0; i < 3; ++i) { s.p[i] = __fmaf_rn(-pk, s.k[i], s.p[i]); pp = __fmaf_rn(s.p[i], s.p[i], pp); }
            const float ps = rsqrtf(pp);
            for (int i = 0; i < 3; ++i) s.p[i] *= ps;
        }
        // new anchor from small terms: k'.N = sgn * T, T = Ac - sB - 2e + 2q (sB + e)
        const float T = Ac - s.sB - 2.0f * e + 2.0f * q * (s.sB + e);
        if (T < 0.0f) {
            s.A = -Ac + 2.0f * e - 2.0f * q * (s.sB + e);
            s.sgn = -s.sgn;
        } else {
            s.A = T - s.sB;
        }
        segment<GEOM_T, ORD>(L, s);
    }
    return -1;
}

// Work plan: chunks of (job, ray range) claimed by blocks from a global counter.
struct WorkPlan {
    const Launch32 *jobs;                 // device job table, or nullptr for the single job
    const unsigned long long *chunk_begin;// first chunk index of each job (n_jobs + 1 entries)
    int32_t n_jobs;
    uint32_t chunk_rays;
    unsigned long long n_chunks;
    unsigned long long *counter;          // zero before the launch
};

// GEOM >= 0: single-job kernel, parameters read from the launch's constant
// bank; GEOM < 0: the generic batched kernel, the block's job staged in smem.
// EXT (generic kernel only): polarised sources and user-supplied rays.
template <int GEOM, int IRC, bool REC, int OCC, bool EXT = false>
__global__ void __launch_bounds__(kBlockThreads, OCC)
    k_trace_fp32(const __grid_constant__ Launch32 single, const __grid_constant__ WorkPlan W) {
    constexpr bool BATCH = GEOM < 0;
    static_assert(!EXT || BATCH, "the extended kernel is the generic one");
    __shared__ Launch32 sL;
    __shared__ float s_tab[kMdfKnots];
    __shared__ WarpBuf s_buf[kWarpsPerBlock];
    __shared__ float s_pol[EXT ? kWarpsPerBlock : 1][3][EXT ? kBuf : 1];   // buffered polarisations
    __shared__ BlockTally bt;
    __shared__ unsigned long long s_next, s_end, s_chunk;
    __shared__ int s_job;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    WarpBuf &B = s_buf[wid];
    float (*Bp)[EXT ? kBuf : 1] = s_pol[EXT ? wid : 0];
    const Launch32 &L = BATCH ? sL : single;
    int cur_job = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long c = atomicAdd(W.counter, 1ull);
            s_chunk = c;
            if (c < W.n_chunks) {
                int j = 0;
                unsigned long long first = c * (unsigned long long)W.chunk_rays, nj = single.n;
                if (W.jobs) {
                    int lo = 0, hi = W.n_jobs;           // largest j with chunk_begin[j] <= c
                    while (hi - lo > 1) { const int m = (lo + hi) >> 1; if (W.chunk_begin[m] <= c) lo = m; else hi = m; }
                    j = lo;
                    first = (c - W.chunk_begin[j]) * (unsigned long long)W.chunk_rays;
                    nj = W.jobs[j].n;
                }
                s_job = j;
                s_next = first;
                s_end = min(first + (unsigned long long)W.chunk_rays, nj);
            }
        }
        __syncthreads();
        if (s_chunk >= W.n_chunks) break;
        const int j = s_job;
        if (j != cur_job) {
            // this block's job changed: load its parameters, then its mosaic table
            if (BATCH) {
                // a single-job launch of the generic kernel stages its parameter block
                const uint32_t *src = (const uint32_t *)(W.jobs ? &W.jobs[j] : &single);
                uint32_t *dst = (uint32_t *)&sL;
                for (int i = threadIdx.x; i < (int)(sizeof(Launch32) / 4); i += blockDim.x) dst[i] = src[i];
                __syncthreads();
            }
            for (int i = threadIdx.x; i < kMdfKnots; i += blockDim.x) s_tab[i] = L.tab[i];
            cur_job = j;
        }
        for (int i = threadIdx.x; i < kTallyN; i += blockDim.x) bt.t[i] = 0u;
        if (threadIdx.x == 0) { bt.coll = 0ull; bt.emit = 0ull; bt.miss = 0ull; }
        if (lane == 0) B.count = 0;
        __syncthreads();

        Lane s;
        bool alive = false;
        bool more = true;
        unsigned long long my_coll = 0, my_emit = 0, my_miss = 0;
        for (;;) {
            const unsigned idle = __ballot_sync(0xffffffffu, !alive);
            const int n_idle = __popc(idle);
            if (n_idle == 32 && !more && B.count == 0) break;
            if (n_idle >= L.refill || (n_idle > 0 && !more) || n_idle == 32) {
                while (more && B.count < n_idle && B.count < kSpawnBelow) {
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(&s_next, 32ull);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    const unsigned long long end = s_end;
                    if (base >= end) { more = false; break; }
                    const unsigned long long id = base + lane;
                    float x[3], k[3], A = 0.f, sB = 0.f, mu0 = 0.f, qr = 0.f, inv_ws = 1.f, E32 = 0.f;
                    float pv[3] = {0.f, 0.f, 0.f};
                    float oA[HEART_MAX_ORDERS] = {0.f, 0.f, 0.f, 0.f}, osB[HEART_MAX_ORDERS] = {0.f, 0.f, 0.f, 0.f};
                    int nb = 0, nbm = 0;
                    bool hit = false;
                    if (id < end) {
                        ++my_emit;
                        if (EXT && L.user) {
                            hit = spawn_user<GEOM>(L, id, x, k, pv, A, sB, mu0, qr, inv_ws, E32, nb,
                                                   EXT ? oA : nullptr, EXT ? osB : nullptr, EXT ? &nbm : nullptr);
                        } else {
                            hit = spawn<GEOM>(L, L.offset + id, x, k, A, sB, mu0, qr, inv_ws, E32, nb,
                                              EXT ? oA : nullptr, EXT ? osB : nullptr, EXT ? &nbm : nullptr);
                            if (EXT && L.pol_on) project_pol32(L, k, pv);
                        }
                        if (!hit) {
                            ++my_miss;
                            if (REC) write_miss_record(L, L.offset + id, x, k, E32, pv);
                        }
                    }
                    const unsigned hm = __ballot_sync(0xffffffffu, hit);
                    if (hit && EXT && L.n_ord > 1) {
                        // several orders: the buffer's segment fields carry the anchors and
                        // sines of orders 1-3 and the no-Bragg mask; the walking lane
                        // prepares the entry segment of all orders when it pops the ray
                        const int slot = B.count + __popc(hm & lt_mask);
                        for (int i = 0; i < 3; ++i) { B.x[i][slot] = x[i]; B.k[i][slot] = k[i]; Bp[i][slot] = pv[i]; }
                        const uint64_t ray = L.offset + id;
                        B.A[slot] = A;
                        B.sB[slot] = sB;
                        B.rl[slot] = (uint32_t)ray;
                        B.rh[slot] = (uint32_t)(ray >> 32);
                        B.mu0[slot] = mu0;
                        B.E[slot] = E32;
                        B.s_exit[slot] = oA[1];
                        B.inv_mu[slot] = osB[1];
                        B.pa[slot] = oA[2];
                        B.ra[slot] = osB[2];
                        B.qmin[slot] = oA[3];
                        B.pbar[slot] = osB[3];
                        B.face[slot] = nbm;
                    } else if (hit) {
                        // the entry segment: exit face and distance, majorant and thinning bounds
                        Lane t;
                        for (int i = 0; i < 3; ++i) { t.x0[i] = x[i]; t.k[i] = k[i]; }
                        t.A = A;
                        t.sB = sB;
                        t.cB = sqrtf(fmaxf(0.0f, __fmaf_rn(-sB, sB, 1.0f)));
                        t.sgn = -1.0f;                           // entering: k.N < 0
                        t.rho0 = 0.0f;                           // on the front face
                        t.mu0 = mu0;
                        t.qr = qr;
                        t.inv_ws = inv_ws;
                        segment<GEOM>(L, t);
                        const int slot = B.count + __popc(hm & lt_mask);
                        for (int i = 0; i < 3; ++i) { B.x[i][slot] = x[i]; B.k[i][slot] = k[i]; }
                        const uint64_t ray = L.offset + id;
                        B.A[slot] = A;
                        B.sB[slot] = sB;
                        B.rl[slot] = (uint32_t)ray;
                        B.rh[slot] = (uint32_t)(ray >> 32);
                        B.mu0[slot] = mu0;
                        B.qr[slot] = qr;
                        B.inv_ws[slot] = inv_ws;
                        B.E[slot] = E32;
                        B.nb[slot] = nb;
                        B.s_exit[slot] = t.s_exit;
                        B.face[slot] = t.face;
                        B.inv_mu[slot] = t.inv_mu;
                        B.pa[slot] = t.pa;
                        B.ra[slot] = t.ra;
                        B.qmin[slot] = t.qmin;
                        B.pbar[slot] = t.pbar;
                        B.w0[slot] = t.w0;
                        B.w1[slot] = t.w1;
                        B.pbarB[slot] = t.pbarB;
                        if (EXT) for (int i = 0; i < 3; ++i) Bp[i][slot] = pv[i];
                    }
                    __syncwarp();
                    if (lane == 0) B.count += __popc(hm);
                    __syncwarp();
                    if (base + 32 >= end) more = false;
                }
                const int avail = B.count;
                const int rank = __popc(idle & lt_mask);
                if (!alive && rank < avail) {
                    const int slot = avail - 1 - rank;
                    for (int i = 0; i < 3; ++i) { s.x0[i] = B.x[i][slot]; s.k[i] = B.k[i][slot]; }
                    s.A = B.A[slot];
                    s.sB = B.sB[slot];
                    s.rl = B.rl[slot];
                    s.rh = B.rh[slot];
                    s.mu0 = B.mu0[slot];
                    s.qr = B.qr[slot];
                    s.inv_ws = B.inv_ws[slot];
                    s.E = B.E[slot];
                    s.no_bragg = B.nb[slot];
                    s.s_exit = B.s_exit[slot];
                    s.face = B.face[slot];
                    s.inv_mu = B.inv_mu[slot];
                    s.pa = B.pa[slot];
                    s.ra = B.ra[slot];
                    s.qmin = B.qmin[slot];
                    s.pbar = B.pbar[slot];
                    s.w0 = B.w0[slot];
                    s.w1 = B.w1[slot];
                    s.pbarB = B.pbarB[slot];
                    s.inv_1mpa = s.pa < 1.0f ? 1.0f / (1.0f - s.pa) : 0.0f;
                    s.pa_thr = s.pa >= 1.0f ? 0xFFFFFFFFu
                                            : __float2uint_ru(fminf(s.pa * 4294967296.0f, 4294967040.0f));
                    s.cB = sqrtf(fmaxf(0.0f, __fmaf_rn(-s.sB, s.sB, 1.0f)));
                    s.sgn = -1.0f;                           // entering: k.N < 0
                    s.rho0 = 0.0f;                           // on the front face
                    s.call = 2u;
                    s.nrefl = 0;
                    s.ncoll = 0;
                    s.pol = false;
                    if (EXT) {
                        for (int i = 0; i < 3; ++i) s.p[i] = Bp[i][slot];
                        s.pol = s.p[0] != 0.0f || s.p[1] != 0.0f || s.p[2] != 0.0f;
                    }
                    if (EXT && L.n_ord > 1) {
                        const float oa[4] = {s.A, B.s_exit[slot], B.pa[slot], B.qmin[slot]};
                        const float os[4] = {s.sB, B.inv_mu[slot], B.ra[slot], B.pbar[slot]};
                        start_orders(L, s, oa, os, B.face[slot]);
                        segment<GEOM, true>(L, s);            // the entry segment of every order
                    } else {
                        segment_consts<GEOM>(L, s);           // the rest of the entry segment was prepared
                    }
                    alive = true;
                }
                __syncwarp();
                if (lane == 0) B.count = avail - min(avail, n_idle);
                __syncwarp();
            }
            if (alive) {
                const int oc = step<GEOM, IRC, EXT, EXT>(L, s, s_tab);
                if (oc >= 0) {
                    my_coll += (unsigned long long)s.ncoll;
                    finish<REC, EXT>(L, s, oc, bt);
                    alive = false;
                }
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            my_coll += __shfl_down_sync(0xffffffffu, my_coll, off);
            my_emit += __shfl_down_sync(0xffffffffu, my_emit, off);
            my_miss += __shfl_down_sync(0xffffffffu, my_miss, off);
        }
        if (lane == 0) {
            atomicAdd(&bt.coll, my_coll);
            atomicAdd(&bt.emit, my_emit);
            atomicAdd(&bt.miss, my_miss);
        }
        __syncthreads();
        // flush this chunk's tallies to the job
        unsigned long long *T = L.tally;
        for (int i = threadIdx.x; i < kTallyN; i += blockDim.x) {
            unsigned long long v = bt.t[i];
            if (i == T_COLLISIONS) v = bt.coll;
            if (i == T_EMITTED) v = bt.emit;
            if (i == T_MISS) v = bt.miss;
            if (v) atomicAdd(&T[i], v);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Two-pass ("wavefront") trace of one job, for image traces of one reflection
// order without polarisation or user rays.  With the thinned sampler a ray
// makes about one tentative collision, so the per-ray work (source, entry,
// preparing the entry segment) weighs as much as the walk: doing it in a
// separate pass, one thread per ray at full occupancy, and handing the hits
// to the walk pass through a compacted queue in global memory (chunks of
// kWaveCap rays, which keeps the queue near the L2) spends far fewer issue
// slots than spawning inside the walk loop.  Both passes run the same device
// functions as the persistent kernel, so every ray is traced identically.
// ---------------------------------------------------------------------------
// a prepared hit: one 96-byte record of six 16-byte words, written and read
// with vector stores and loads (consecutive lanes touch consecutive records):
//   [x0 x1 x2 k0] [k1 k2 A sB] [mu0 qr inv_ws E] [s_exit inv_mu pa ra]
//   [qmin pbar ray_lo ray_hi] [w0 face|no_bragg<<8 w1 pbarB]
// and for a polarised source a seventh word [p0 p1 p2 -] (112-byte records)
template <bool POL>
__device__ __forceinline__ float4 *wave_rec(const WaveBuf &B, size_t slot) {
    return (float4 *)B.base + slot * (size_t)(POL ? kWaveRec16 + 1 : kWaveRec16);
}

// pass 1: one thread per ray of [first, first + count), in two phases.  First
// every thread draws its ray's geometry and tests the entry; the rays that
// entered are compacted through shared memory (block offsets from a scan of
// the warps' hit counts, one global atomic per block reserving their queue
// slots).  Then the first `hits` threads of the block take one entered ray
// each and do the rest of its set-up with full warps: energy, Bragg anchor,
// rates and the entry segment, and write its record.  (A counter that every
// warp of the grid incremented serialised the pass; preparing the segments in
// the threads that drew the rays left 59 % of their lanes idle.)  A ray whose
// energy is not positive and finite is queued as a dead record (no_bragg = 2)
// that the walk counts as a miss.  Emitted rays and misses are tallied by the
// walk pass from count and the queue length.
constexpr int kSpawnThreads = 256, kSpawnWarps = kSpawnThreads / 32;
// staged entered rays: sampled sources keep dA (the set-up draws the energy's
// Philox block from the ray id); user-supplied rays, set up in full by
// spawn_user, keep A in dA and sB, mu0, qr, inv_ws in u, with E and no_bragg
template <bool POL, bool USER>
struct SpawnStage {
    float x[3][kSpawnThreads], k[3][kSpawnThreads], dA[kSpawnThreads];
    float u[4][USER ? kSpawnThreads : 1];
    uint32_t idx[kSpawnThreads];
    float p[3][POL ? kSpawnThreads : 1];                 // polarisation (polarised sources, user rays)
    float e[USER ? kSpawnThreads : 1];
    int32_t nb[USER ? kSpawnThreads : 1];
};
// ORD: several reflection orders (sampled rays): the record's segment words carry
// orders 1-3's anchors and sines and the no-Bragg mask, and the walk prepares the
// entry segment of every order when it takes the ray
template <int GEOM, bool POL, bool USER, bool ORD = false>
__global__ void __launch_bounds__(kSpawnThreads, (USER || ORD) ? 4 : 8) k_spawn32(const __grid_constant__ Launch32 L,
                                                           const __grid_constant__ WaveBuf B, uint64_t first,
                                                           uint32_t count, unsigned long long *n_hits) {
    static_assert(!USER || POL, "user rays travel with their polarisation word");
    static_assert(!ORD || (POL && !USER), "several orders: the polarised variant, sampled rays");
    __shared__ SpawnStage<POL, USER> sg;
    __shared__ unsigned int s_ofs[kSpawnWarps];
    __shared__ unsigned long long s_base;
    __shared__ unsigned int s_hits;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    {
        float x[3], k[3], dA = 0.0f, pv[3] = {0.0f, 0.0f, 0.0f};
        float uw[4] = {0.f, 0.f, 0.f, 1.f};
        float uE = 0.0f;
        int unb = 0;
        bool hit;
        if (USER) {
            // the ray's own origin, direction, energy and polarisation, entered in FP64
            hit = i < count && spawn_user<GEOM>(L, first + i, x, k, pv, dA, uw[0], uw[1], uw[2], uw[3], uE, unb);
        } else {
            hit = i < count && spawn_entry<GEOM>(L, L.offset + first + i, x, k, dA);
            if (POL && hit) project_pol32(L, k, pv);
        }
        const unsigned hm = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) s_ofs[warp] = __popc(hm);
        __syncthreads();
        if (warp == 0) {
            // exclusive scan of the warps' hit counts, one global atomic for the block
            const unsigned c = lane < kSpawnWarps ? s_ofs[lane] : 0u;
            unsigned inc = c;
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc += y;
            }
            const unsigned total = __shfl_sync(0xffffffffu, inc, 31);
            unsigned long long bs = 0;
            if (lane == 0 && total) bs = atomicAdd(n_hits, (unsigned long long)total);
            if (lane < kSpawnWarps) s_ofs[lane] = inc - c;
            if (lane == 0) { s_base = bs; s_hits = total; }
        }
        __syncthreads();
        if (hit) {
            const unsigned j = s_ofs[warp] + __popc(hm & ((1u << lane) - 1u));
            for (int m = 0; m < 3; ++m) { sg.x[m][j] = x[m]; sg.k[m][j] = k[m]; }
            sg.dA[j] = dA;
            if (USER)
                for (int m = 0; m < 4; ++m) sg.u[m][USER ? j : 0] = uw[m];
            sg.idx[j] = threadIdx.x;
            if (POL)
                for (int m = 0; m < 3; ++m) sg.p[m][POL ? j : 0] = pv[m];
            if (USER) { sg.e[USER ? j : 0] = uE; sg.nb[USER ? j : 0] = unb; }
        }
        __syncthreads();
    }
    const unsigned j = threadIdx.x;
    if (j >= s_hits) return;
    float A = 0.f, sB = 0.f, mu0 = 0.f, qr = 0.f, inv_ws = 1.f, E32 = 0.f;
    int nb = 0, nbm = 0;
    float oA[HEART_MAX_ORDERS] = {0.f, 0.f, 0.f, 0.f}, osB[HEART_MAX_ORDERS] = {0.f, 0.f, 0.f, 0.f};
    bool ok = true;
    if (USER) {
        A = sg.dA[j];
        sB = sg.u[0][USER ? j : 0]; mu0 = sg.u[1][USER ? j : 0];
        qr = sg.u[2][USER ? j : 0]; inv_ws = sg.u[3][USER ? j : 0];
        E32 = sg.e[USER ? j : 0];
        nb = sg.nb[USER ? j : 0];
    } else {
        uint32_t e[4];
        const uint64_t ray = L.offset + first + (uint64_t)blockIdx.x * blockDim.x + sg.idx[j];
        philox_l<(GEOM >= 0)>(L, (uint32_t)ray, (uint32_t)(ray >> 32), 1u, 0u, e);
        ok = spawn_energy(L, e[0], e[1], e[2], e[3], sg.dA[j], A, sB, mu0, qr, inv_ws, E32, nb,
                          ORD ? oA : nullptr, ORD ? osB : nullptr, ORD ? &nbm : nullptr);
    }
    Lane t;
    for (int m = 0; m < 3; ++m) { t.x0[m] = sg.x[m][j]; t.k[m] = sg.k[m][j]; }
    t.s_exit = 0.f; t.inv_mu = 0.f; t.pa = 0.f; t.ra = 0.f; t.qmin = 0.f; t.pbar = 0.f; t.w0 = 0u; t.face = 0;
    t.w1 = 0u; t.pbarB = 0.f;
    if (ORD) {
        t.s_exit = oA[1]; t.inv_mu = osB[1]; t.pa = oA[2]; t.ra = osB[2]; t.qmin = oA[3]; t.pbar = osB[3];
        t.face = nbm;
    } else if (ok) {
        t.A = A;
        t.sB = sB;
        t.cB = sqrtf(fmaxf(0.0f, __fmaf_rn(-sB, sB, 1.0f)));
        t.sgn = -1.0f;                                       // entering: k.N < 0
        t.rho0 = 0.0f;                                       // on the front face
        t.mu0 = mu0;
        t.qr = qr;
        t.inv_ws = inv_ws;
        segment<GEOM>(L, t);
    }
    const uint64_t ray = L.offset + first + (uint64_t)blockIdx.x * blockDim.x + sg.idx[j];
    float4 *r = wave_rec<POL>(B, s_base + j);
    if (POL) r[kWaveRec16] = make_float4(sg.p[0][POL ? j : 0], sg.p[1][POL ? j : 0], sg.p[2][POL ? j : 0], 0.0f);
    r[0] = make_float4(t.x0[0], t.x0[1], t.x0[2], t.k[0]);
    r[1] = make_float4(t.k[1], t.k[2], A, sB);
    r[2] = make_float4(mu0, qr, inv_ws, E32);
    r[3] = make_float4(t.s_exit, t.inv_mu, t.pa, t.ra);
    r[4] = make_float4(t.qmin, t.pbar, __uint_as_float((uint32_t)ray), __uint_as_float((uint32_t)(ray >> 32)));
    r[5] = make_float4(__uint_as_float(t.w0), __int_as_float(t.face | ((ok ? nb : 2) << 8)), __uint_as_float(t.w1),
                       t.pbarB);
}

// Per-ray records of the rays a two-pass trace does not queue (tests): those
// that miss the crystal or draw no valid energy.  The same source and entry
// functions as the spawn pass, one thread per ray; the walk pass writes the
// records of the queued rays.
template <int GEOM, bool POL, bool USER>
__global__ void __launch_bounds__(256) k_miss_rec32(const __grid_constant__ Launch32 L, uint64_t first,
                                                    uint32_t count) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float x[3], k[3], pv[3] = {0.0f, 0.0f, 0.0f}, A = 0.f, sB = 0.f, mu0 = 0.f, qr = 0.f, inv_ws = 1.f, E32 = 0.f;
    int nb = 0;
    bool ok;
    if (USER) {
        ok = spawn_user<GEOM>(L, first + i, x, k, pv, A, sB, mu0, qr, inv_ws, E32, nb);
    } else {
        ok = spawn<GEOM>(L, L.offset + first + i, x, k, A, sB, mu0, qr, inv_ws, E32, nb);
        if (POL) project_pol32(L, k, pv);
    }
    if (!ok) write_miss_record(L, L.offset + first + i, x, k, E32, pv);
}

// pass 2: a persistent grid walks the queued hits; idle lanes take the next
// ones (warp-aggregated) once at least `refill` lanes of the warp are idle.
// REC: also write each queued ray's record (tests; the same device functions,
// so the same decisions as the variants without records)
template <int GEOM, int IRC, int OCC, bool POL, bool ORD = false, bool REC = false>
__global__ void __launch_bounds__(kBlockThreads, OCC)
    k_walk32(const __grid_constant__ Launch32 L, const __grid_constant__ WaveBuf B,
             const unsigned long long *n_hits, unsigned long long *head, uint32_t count) {
    __shared__ float s_tab[kMdfKnots];
    __shared__ BlockTally bt;
    for (int i = threadIdx.x; i < kMdfKnots; i += blockDim.x) s_tab[i] = L.tab[i];
    for (int i = threadIdx.x; i < kTallyN; i += blockDim.x) bt.t[i] = 0u;
    if (threadIdx.x == 0) { bt.coll = 0ull; bt.emit = 0ull; bt.miss = 0ull; }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned long long nh = *(volatile const unsigned long long *)n_hits;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the chunk's emitted rays and misses (every ray of the chunk that is not queued missed)
        atomicAdd(&L.tally[T_EMITTED], (unsigned long long)count);
        atomicAdd(&L.tally[T_MISS], (unsigned long long)count - nh);
    }
    // Queue slots are claimed 32 at a time, one claim ahead: lane 0 holds the current
    // claim's first slot (cb) and the next one's (nb); a refill hands out the current
    // claim's slots from position cpos on and, past its end, the next claim's; when the
    // current claim is used up the next becomes current and a new claim is issued, whose
    // atomic completes long before its slots are handed out.  (Queue indices of a chunk
    // fit in 32 bits.)
    constexpr uint32_t kClaim = 32;
    unsigned int *head32 = (unsigned int *)head;      // the low word of the chunk's head counter
    uint32_t cb = 0, nb = 0, cpos = 0;
    if (!ORD && lane == 0) {
        cb = atomicAdd(head32, 2u * kClaim);
        nb = cb + kClaim;
    }
    const uint32_t nh32 = (uint32_t)nh;
    Lane s;
    bool alive = false, more = ORD || __shfl_sync(0xffffffffu, cb, 0) < nh32;
    uint32_t my_coll = 0, my_dead = 0;         // per lane: far below 2^32 in one launch
    for (;;) {
        const unsigned idle = __ballot_sync(0xffffffffu, !alive);
        const uint32_t n_idle = __popc(idle);
        if (!more && n_idle == 32) break;
        if (more && (n_idle >= (uint32_t)L.refill || n_idle == 32)) {
            unsigned long long slot;
            if constexpr (ORD) {
                // several orders: one claim per refill (the claim ahead measured slower here:
                // 6.8e9 against 8.3e9 rays/s with three orders)
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(head, (unsigned long long)n_idle);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base + n_idle >= nh) more = false;
                slot = base + __popc(idle & lt_mask);
            } else {
                const uint32_t cbu = __shfl_sync(0xffffffffu, cb, 0), nbu = __shfl_sync(0xffffffffu, nb, 0);
                const uint32_t rank = __popc(idle & lt_mask), left = kClaim - cpos;
                slot = rank < left ? cbu + cpos + rank : nbu + (rank - left);
                {
                    // the next claim's records into L1 ahead of their loads: one line per lane
                    // (the claim's 32 records span 24 lines, 28 with the polarisation word)
                    constexpr uint32_t kLines = (kClaim * 16u * (POL ? kWaveRec16 + 1 : kWaveRec16)) / 128u;
                    const char *q = (const char *)wave_rec<POL>(B, nbu) + 128u * lane;
                    if (lane < kLines && nbu < nh32 && q < (const char *)wave_rec<POL>(B, B.cap))
                        asm volatile("prefetch.global.L1 [%0];" ::"l"(q));
                }
                cpos += n_idle;
                uint32_t next = cbu + cpos;
                if (cpos >= kClaim) {
                    cpos -= kClaim;
                    next = nbu + cpos;
                    if (lane == 0) {
                        cb = nb;
                        nb = atomicAdd(head32, kClaim);
                    }
                }
                if (next >= nh32) more = false;
            }
            if (!alive && slot < nh) {
                const float4 *r = wave_rec<POL>(B, slot);
                const float4 r0 = __ldcs(r), r1 = __ldcs(r + 1), r2 = __ldcs(r + 2), r3 = __ldcs(r + 3),
                             r4 = __ldcs(r + 4), r5 = __ldcs(r + 5);
                if (POL) {
                    const float4 r6 = __ldcs(r + kWaveRec16);
                    s.p[0] = r6.x; s.p[1] = r6.y; s.p[2] = r6.z;
                }
                s.x0[0] = r0.x; s.x0[1] = r0.y; s.x0[2] = r0.z; s.k[0] = r0.w;
                s.k[1] = r1.x; s.k[2] = r1.y; s.A = r1.z; s.sB = r1.w;
                s.mu0 = r2.x; s.qr = r2.y; s.inv_ws = r2.z; s.E = r2.w;
                s.s_exit = r3.x; s.inv_mu = r3.y; s.pa = r3.z; s.ra = r3.w;
                s.qmin = r4.x; s.pbar = r4.y; s.rl = __float_as_uint(r4.z); s.rh = __float_as_uint(r4.w);
                s.w0 = __float_as_uint(r5.x); s.face = __float_as_int(r5.y) & 0xff;
                s.no_bragg = __float_as_int(r5.y) >> 8; s.w1 = __float_as_uint(r5.z); s.pbarB = r5.w;
                if (s.no_bragg == 2) {
                    ++my_dead;                                // no valid energy: a miss, nothing to walk
                } else {
                    s.inv_1mpa = s.pa < 1.0f ? 1.0f / (1.0f - s.pa) : 0.0f;
                    s.pa_thr = s.pa >= 1.0f ? 0xFFFFFFFFu
                                            : __float2uint_ru(fminf(s.pa * 4294967296.0f, 4294967040.0f));
                    s.cB = sqrtf(fmaxf(0.0f, __fmaf_rn(-s.sB, s.sB, 1.0f)));
                    s.sgn = -1.0f;
                    s.rho0 = 0.0f;
                    s.call = 2u;
                    s.nrefl = 0;
                    s.ncoll = 0;
                    s.pol = POL && (s.p[0] != 0.0f || s.p[1] != 0.0f || s.p[2] != 0.0f);
                    if (ORD) {
                        // every order's rates and the entry segment of all orders
                        const float oa[4] = {s.A, r3.x, r3.z, r4.x}, os[4] = {s.sB, r3.y, r3.w, r4.y};
                        start_orders(L, s, oa, os, __float_as_int(r5.y) & 0xff);
                        segment<GEOM, true>(L, s);
                    } else {
                        segment_consts<GEOM>(L, s);
                    }
                    alive = true;
                }
            }
        }
        if (alive) {
            const int oc = step<GEOM, IRC, POL, ORD>(L, s, s_tab);
            if (oc >= 0) {
                my_coll += (uint32_t)s.ncoll;
                finish<REC, POL>(L, s, oc, bt);
                alive = false;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        my_coll += __shfl_down_sync(0xffffffffu, my_coll, off);
        my_dead += __shfl_down_sync(0xffffffffu, my_dead, off);
    }
    if (lane == 0) {
        atomicAdd(&bt.coll, (unsigned long long)my_coll);
        if (my_dead) atomicAdd(&L.tally[T_MISS], (unsigned long long)my_dead);
    }
    __syncthreads();
    unsigned long long *T = L.tally;
    for (int i = threadIdx.x; i < kTallyN; i += blockDim.x) {
        const unsigned long long v = i == T_COLLISIONS ? bt.coll : (unsigned long long)bt.t[i];
        if (v && i != T_EMITTED && i != T_MISS) atomicAdd(&T[i], v);
    }
}

// Device functions of the FP32 kernels evaluated on arrays (tests):
// 0: acos_ratio(x, y, 1 / y); 1: the rocking curve R(x) / R_max (irc_rel32);
// 2: its upper bound over |x'| >= x used by the early rejection (irc_bound32);
// 3: the arc measure bound arc_bound(x, y, z, 1 / z); 4: the measure arc_sample
// takes for that interval, its arc length over pi
__global__ void k_check_functions(const __grid_constant__ Launch32 L, int which, const float *x, const float *y,
                                  const float *z, float *out, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        float r;
        if (which == 0) r = acos_ratio(x[i], y[i], 1.0f / y[i]);
        else if (which == 1) r = irc_rel32<-1>(L, x[i]);
        else if (which == 2) r = irc_bound32<-1>(L, x[i]);
        else if (which == 3) r = arc_bound(x[i], y[i], z[i], 1.0f / z[i]);
        else {
            float st, len;
            arc_piece(x[i], y[i], z[i], 1.0f / z[i], st, len);
            r = len * 0.318309886f;
        }
        out[i] = r;
    }
}

// ---------------------------------------------------------------------------
// host side: crystal-frame parameters, small-quantity anchors and launch
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
    double o[3], ax[3], b1[3], b2[3];
    to_local(S, P.origin, o, true);
    to_local(S, P.ax, ax, false);
    to_local(S, P.b1, b1, false);
    to_local(S, P.b2, b2, false);
    for (int i = 0; i < 3; ++i) {
        L.o[i] = (float)o[i];
        L.ax[i] = (float)ax[i];
        L.b1[i] = (float)b1[i];
        L.b2[i] = (float)b2[i];
    }
    L.omc = (float)P.one_minus_cos_max;
    L.sig1 = (float)P.sig1;
    L.sig2 = (float)P.sig2;
    // the reference direction's normal component: flat N (local z), cylinder axis (local x)
    const double a_n = S.geometry == HEART_FLAT ? ax[2] : ax[0];
    L.a_n = (float)a_n;
    const double axis_sine = std::sqrt(std::fmax(0.0, 1.0 - a_n * a_n));   // cylinder: |k.N| of the axis ray
    L.c_a = (float)axis_sine;
    const double cs = std::cos(S.irc_shift), sn = std::sin(S.irc_shift);
    L.n_irc_e = S.n_irc_e;
    for (int i = 0; i < S.n_irc_e; ++i) {
        L.irc_e[i] = (float)S.irc_e[i];
        L.irc_ws[i] = (float)S.irc_ws[i];
        L.irc_sh[i] = (float)S.irc_sh[i];
    }
    L.shift0 = S.irc_shift;
    // reflection orders: order 0's multiple, K ratio and width ratio enter the
    // single-order fields (sin aB on d / m_0, K_0, widths w_0 times the described)
    const double m0 = (double)S.ord_m[0];
    L.n_ord = S.n_orders;
    L.xs_on = S.n_irc_e > 0;
    for (int h = 0; h < S.n_orders; ++h) {
        L.ord_r[h] = (float)(S.ord_m[h] / m0);
        L.ord_rd[h] = S.ord_m[h] / m0;
        L.ord_k2[h] = (float)(S.K * S.ord_k[h] * S.K * S.ord_k[h]);
        L.ord_iw[h] = (float)(1.0 / S.ord_w[h]);
        if (S.ord_w[h] != 1.0) L.xs_on = 1;
    }
    L.n_comp = P.n_comp;
    for (int i = 0; i < P.n_comp; ++i) {
        // first word w with (w + 1/2) 2^-32 >= cumw
        const double thr = std::ceil(P.cumw[i] * 4294967296.0 - 0.5);
        L.comp_thr[i] = thr >= 4294967295.0 ? 0xFFFFFFFFu : (thr <= 0 ? 0u : (uint32_t)thr);
        L.kind[i] = P.kind[i];
        double e_ref = P.e0[i];
        switch (P.kind[i]) {
        case HEART_SRC_INV_E:
            e_ref = std::sqrt(P.lo[i] * P.hi[i]);
            L.half_ln[i] = (float)std::log(P.hi[i] / P.lo[i]);
            break;
        case HEART_SRC_UNIFORM:
            e_ref = 0.5 * (P.lo[i] + P.hi[i]);
            L.width[i] = (float)(P.hi[i] - P.lo[i]);
            break;
        case HEART_SRC_TABLE: e_ref = P.tab_mean; break;
        default:
            L.width[i] = (float)P.width[i];
        }
        L.e_ref[i] = (float)e_ref;
        L.lF0[i] = (float)P.lorentz_F0[i];
        const double s0 = m0 * 12.398419843320026 / (2.0 * S.d_A * e_ref);
        L.sB_raw[i] = (float)s0;
        const double c0 = s0 < 1.0 ? std::sqrt(1.0 - s0 * s0) : 0.0;
        L.cB_raw[i] = (float)c0;
        // the peak shift at the reference energy: Delta_M plus the energy table's shift there
        double ws_ref = 1.0, sh_ref = 0.0;
        if (S.n_irc_e > 0) irc_energy64(S, e_ref, ws_ref, sh_ref);
        L.sh_ref[i] = (float)sh_ref;
        const double csi = S.n_irc_e > 0 ? std::cos(S.irc_shift + sh_ref) : cs;
        const double sni = S.n_irc_e > 0 ? std::sin(S.irc_shift + sh_ref) : sn;
        L.cos_shift[i] = (float)csi;
        L.sin_shift[i] = (float)sni;
        // sin(aB + Delta_M) and the anchor of the cone-axis ray, |a_n| (flat) or the
        // axis sine (cylinder) minus that sine, for every order (order 0 first)
        const double kref = S.geometry == HEART_FLAT ? std::fabs(a_n) : axis_sine;
        for (int h = 0; h < S.n_orders; ++h) {
            const double sh0 = s0 * (S.ord_m[h] / m0), ch0 = sh0 < 1.0 ? std::sqrt(1.0 - sh0 * sh0) : 0.0;
            const double sBh = sh0 * csi + ch0 * sni;
            L.osB0[h][i] = (float)sBh;
            L.oA0[h][i] = (float)(kref - sBh);
        }
    }
    L.half_d = (float)S.half_d;
    L.half_n = (float)S.half_n;
    L.thick = (float)S.thickness;
    L.R = (float)S.radius;
    L.zc = (float)S.zc;
    L.sphi = (float)S.sphi;
    L.cphi = (float)S.cphi;
    // rocking curve, relative to its maximum
    L.irc_fwhm = (float)S.irc_fwhm;
    L.irc_eta = (float)S.irc_eta;
    L.irc_g = (float)S.irc_g;
    L.irc_c = (float)(4.0 * 0.69314718055994530942 / (S.irc_fwhm * S.irc_fwhm));
    switch (S.irc) {
    case HEART_IRC_DARWIN: L.irc_delta = (float)(1.0 / S.irc_delta); break;
    case HEART_IRC_DARWIN_PRINS:
        L.irc_delta = (float)(1.0 / S.irc_delta);
        L.irc_gnorm = (float)(1.0 / (S.irc_max * S.irc_norm));   // 1 / max R(y)
        break;
    case HEART_IRC_PSEUDO_VOIGT: {
        const double F = S.irc_fwhm, eta = S.irc_eta, pi = 3.14159265358979323846;
        const double L0 = 2.0 / (pi * F), G0 = std::sqrt(4.0 * 0.69314718055994530942 / pi) / F;
        L.irc_eta = (float)(eta * L0);            // weights of the peak-relative shapes
        L.irc_g = (float)((1.0 - eta) * G0);
        L.irc_gnorm = (float)(1.0 / S.irc_max);
        break;
    }
    default: break;
    }
    L.labs = (float)S.labs;
    L.labs_ref = (float)S.labs_ref;
    L.labs_pow = (float)S.labs_pow;
    L.K2 = (float)(S.K * S.ord_k[0] * S.K * S.ord_k[0]);
    L.irc_max = (float)S.irc_max;
    L.mdf = S.mdf;
    L.none_fac = (float)S.none_fac;
    L.w_a2 = (float)S.w_a2;
    L.w_c = (float)S.w_c;
    L.w_wl = (float)S.w_wl;
    L.w_wg = (float)S.w_wg;
    L.w_b = (float)S.w_b;
    L.w_qmax = (float)S.w_qmax;
    L.none_qv = (float)S.none_qv;
    L.max_refl = S.max_refl;
    L.max_coll = S.max_coll;
    double D0[3], eu[3], ev[3], nd[3];
    to_local(S, S.D0, D0, true);
    to_local(S, S.eu, eu, false);
    to_local(S, S.ev, ev, false);
    to_local(S, S.nd, nd, false);
    for (int i = 0; i < 3; ++i) {
        L.D0[i] = (float)D0[i];
        L.eu[i] = (float)eu[i];
        L.ev[i] = (float)ev[i];
        L.nd[i] = (float)nd[i];
    }
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
    uint32_t a = L.k0, b = L.k1;
    for (int r = 0; r < 10; ++r) {
        L.rk0[r] = a;
        L.rk1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    L.sampler = S.sampler;
    L.vstar = (float)S.vstar;
    L.xstar = (float)S.xstar;
    L.hx2 = (float)(2.0 * std::sin(0.5 * S.xstar) * std::sin(0.5 * S.xstar));
    L.sx = (float)std::sin(S.xstar);
    L.refill = g_tune.refill;
    L.geometry = S.geometry;
    L.irc_kind = S.irc;
    L.tab = S.mdf32;
    L.qgrid = S.qgrid;
    {
        const double q2 = std::exp2(kBandJ2 / 8.0 - 48.0);
        L.band_w2 = S.band_w2;
        L.band_q2 = std::nextafter((float)q2, 1.0f);
        L.band_is2 = std::nextafter((float)(1.0 / std::sqrt(q2 * (2.0 - q2))), 0.0f);
        L.band_is1 = S.band_is1;
        L.band_t2 = std::nextafter((float)std::sqrt(q2 / (2.0 - q2)), 1.0f);
    }
    const double *a0 = S.geometry == HEART_FLAT ? S.ed : S.ax;
    const double *a1 = S.geometry == HEART_FLAT ? S.en : S.cc;
    const double *a2 = S.geometry == HEART_FLAT ? S.N : S.ww;
    for (int i = 0; i < 3; ++i) { L.fc[i] = S.c[i]; L.fa[0][i] = a0[i]; L.fa[1][i] = a1[i]; L.fa[2][i] = a2[i]; }
    for (int r = 0; r < 3; ++r)
        for (int i = 0; i < 3; ++i) L.faf[r][i] = (float)L.fa[r][i];
    L.inv_Rd = L.R > 0.0f ? 1.0 / (double)L.R : 0.0;     // the radius the FP32 walk uses
    L.pol_on = P.pol_on;
    L.user = P.user;
    if (P.pol_on && !P.user) {
        double pl[3];
        to_local(S, P.pol, pl, false);
        for (int i = 0; i < 3; ++i) L.pol[i] = (float)pl[i];
    }
    L.hc_2d = m0 * 12.398419843320026 / (2.0 * S.d_A);       // sin aB of order 0 times E
    L.cs_shift = cs;
    L.sn_shift = sn;
    for (int i = 0; i < 10; ++i) L.ray[i] = P.ray[i];
    L.n_tab = P.n_tab;
    L.tab_thr = P.tab_thr;
    L.tab_off = P.tab_off;
    L.tab_inv = P.tab_inv;
    L.tab_dE = P.tab_dE;
    L.tab_w = P.tab_w;
}

template <int GEOM, int IRC, bool REC, int OCC, bool EXT = false>
static void launch_occ(const Launch32 &L, const WorkPlan &W, cudaStream_t st, uint64_t n_chunks) {
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_fp32<GEOM, IRC, REC, OCC, EXT>, kBlockThreads,
                                                      0);
        if (per_sm < 1) per_sm = 1;
    }
    const uint64_t cap = (uint64_t)per_sm * (uint64_t)num_sms();
    const int blocks = (int)(n_chunks < cap ? n_chunks : cap);
    if (blocks > 0) k_trace_fp32<GEOM, IRC, REC, OCC, EXT><<<blocks, kBlockThreads, 0, st>>>(L, W);
}

template <int GEOM, int IRC, bool REC>
static void launch_t(const Launch32 &L, const WorkPlan &W, cudaStream_t st) {
    // records are a test path: one occupancy variant
    if constexpr (!REC) {
        if (g_tune.blocks_per_sm <= 5) {
            launch_occ<GEOM, IRC, REC, 5>(L, W, st, W.n_chunks);
            return;
        }
    }
    launch_occ<GEOM, IRC, REC, 6>(L, W, st, W.n_chunks);
}

// resident blocks of the launch shape in use (for chunk sizing)
static int resident_blocks() {
    static int per_sm[2] = {0, 0};
    const int v = g_tune.blocks_per_sm <= 5 ? 1 : 0;
    if (per_sm[v] == 0) {
        if (v) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[v], k_trace_fp32<-1, -1, false, 5>, kBlockThreads, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[v], k_trace_fp32<-1, -1, false, 6>, kBlockThreads, 0);
        if (per_sm[v] < 1) per_sm[v] = 1;
    }
    return per_sm[v] * num_sms();
}

// rays per work item: about eight items per resident block, a power of two
// between 2^12 and the tuned maximum, so the last wave of items is short
// work items of about 1/8 of a resident block's share of the launch, a power of two from 512 rays
// (small launches, e.g. a served job alone in its round, still spread over the SMs) up to the tuned maximum
static uint32_t chunk_for(uint64_t total_rays) {
    const uint64_t target = total_rays / ((uint64_t)resident_blocks() * 8ull);
    uint32_t c = 512u;
    while ((uint64_t)c * 2 <= target && c * 2 <= g_tune.chunk_rays) c *= 2;
    return c;
}

// ext: some job is polarised or reads user rays -> the extended generic kernel
template <bool REC>
static heart_status dispatch(const Launch32 &L, const WorkPlan &W, cudaStream_t st, bool generic, bool ext) {
    if (W.n_chunks == 0) return HEART_OK;
    if (ext) {
        launch_occ<-1, -1, REC, 6, true>(L, W, st, W.n_chunks);
    } else if (generic || L.irc_kind == HEART_IRC_NONE) {
        // no rocking curve: the generic kernel's run-time branch (rare option, no own instantiation)
        launch_t<-1, -1, REC>(L, W, st);
    } else {
#define HEART_IRC_CASES(G)                                                                    \
    switch (L.irc_kind) {                                                                     \
    case HEART_IRC_DARWIN: launch_t<G, HEART_IRC_DARWIN, REC>(L, W, st); break;              \
    case HEART_IRC_DARWIN_PRINS: launch_t<G, HEART_IRC_DARWIN_PRINS, REC>(L, W, st); break;  \
    case HEART_IRC_PSEUDO_VOIGT: launch_t<G, HEART_IRC_PSEUDO_VOIGT, REC>(L, W, st); break;  \
    case HEART_IRC_GAUSSIAN: launch_t<G, HEART_IRC_GAUSSIAN, REC>(L, W, st); break;          \
    case HEART_IRC_LORENTZIAN: launch_t<G, HEART_IRC_LORENTZIAN, REC>(L, W, st); break;      \
    default: launch_t<G, HEART_IRC_BOX, REC>(L, W, st); break;                                \
    }
        if (L.geometry == HEART_FLAT) { HEART_IRC_CASES(HEART_FLAT) } else { HEART_IRC_CASES(HEART_CYL_VON_HAMOS) }
#undef HEART_IRC_CASES
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "FP32 kernel launch");
    return HEART_OK;
}

static heart_status launch_single(const SpecParams &S, const SourceParams &P, uint64_t n, uint64_t seed,
                                  uint64_t offset, void *img, unsigned long long *scratch, heart_ray_record *rec,
                                  cudaStream_t st, const QeParams *qe) {
    if (n == 0) return HEART_OK;
    Launch32 L;
    make_launch32(S, P, n, seed, offset, L);
    L.img = img;
    L.tally = scratch;
    L.rec = rec;
    if (qe) {
        L.eimg = qe->eimg;
        L.n_qe = qe->n;
        for (int i = 0; i < qe->n; ++i) { L.qe_e[i] = (float)qe->keV[i]; L.qe_v[i] = (float)qe->qe[i]; }
    }
    WorkPlan W;
    std::memset(&W, 0, sizeof W);
    W.n_jobs = 1;
    W.chunk_rays = chunk_for(n);
    W.n_chunks = (n + W.chunk_rays - 1) / W.chunk_rays;
    W.counter = scratch + kCounterWord;
    const bool ext = L.pol_on || L.user || L.n_ord > 1;
    return rec ? dispatch<true>(L, W, st, false, ext) : dispatch<false>(L, W, st, false, ext);
}

// the current device's side stream and fork / join events of the two-pass
// trace (created with its hit queue; used while the queue is leased)
static void wave_side(cudaStream_t *side, cudaEvent_t *fork, cudaEvent_t *join);

template <int GEOM, int IRC, bool POL = false, bool USER = false, bool ORD = false, bool REC = false>
static heart_status launch_wave_t(const Launch32 &L, const WaveBuf &B, uint64_t n, unsigned long long *ctr,
                                  cudaStream_t st) {
    // launch bound of 6 blocks per SM (up to 80 registers): the benchmark's variant then
    // uses 72 and 7 blocks still fit (the grid follows the occupancy query); its code ran
    // 0.6 % faster than under a bound of 7 and 0.4 % faster than under 8 (64 registers)
    constexpr int OCC = 6;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk32<GEOM, IRC, OCC, POL, ORD, REC>, kBlockThreads,
                                                      0);
        if (per_sm < 1) per_sm = 1;
    }
    const int walk_blocks = per_sm * num_sms();
    const uint64_t chunks = (n + B.cap - 1) / B.cap;
    // consecutive chunks alternate between the queue's two buffers and between the caller's
    // stream and a side stream, so a chunk's spawn pass fills the SMs that the previous
    // chunk's walk pass frees as it drains; each stream keeps its own chunks in order (a
    // buffer is reused two chunks later, on the same stream)
    WaveBuf Bs[2] = {B, B};
    Bs[1].base = (char *)B.base + wave_buffer_bytes(B.cap);
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    if (chunks > 1) wave_side(&side, &fork, &join);
    const bool two = side && fork && join;
    cudaError_t e = cudaSuccess;
    for (uint64_t c = 0; c < chunks; ++c) {
        const uint64_t g = c % kWaveGroup;
        if (g == 0) {
            // the counters of a group of chunks: both streams are done with the previous group
            if (two && c > 0) {
                if ((e = cudaEventRecord(join, side)) != cudaSuccess) return cuda_fail(e, "two-pass join");
                if ((e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess) return cuda_fail(e, "two-pass join");
            }
            const uint64_t left = chunks - c < (uint64_t)kWaveGroup ? chunks - c : (uint64_t)kWaveGroup;
            e = cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned long long) * left, st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync hit counters");
            if (two) {
                if ((e = cudaEventRecord(fork, st)) != cudaSuccess) return cuda_fail(e, "two-pass fork");
                if ((e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess) return cuda_fail(e, "two-pass fork");
            }
        }
        unsigned long long *cc = ctr + 2 * g;
        const uint64_t first = c * B.cap;
        const uint32_t count = (uint32_t)(n - first < B.cap ? n - first : B.cap);
        const int b = two ? (int)(c & 1) : 0;
        cudaStream_t sc = b ? side : st;
        k_spawn32<GEOM, POL, USER, ORD><<<(count + kSpawnThreads - 1) / kSpawnThreads, kSpawnThreads, 0, sc>>>(
            L, Bs[b], first, count, cc);
        if (REC) k_miss_rec32<GEOM, POL, USER><<<(count + 255) / 256, 256, 0, sc>>>(L, first, count);
        k_walk32<GEOM, IRC, OCC, POL, ORD, REC><<<walk_blocks, kBlockThreads, 0, sc>>>(L, Bs[b], cc, cc + 1, count);
    }
    if (two) {
        if ((e = cudaEventRecord(join, side)) != cudaSuccess) return cuda_fail(e, "two-pass join");
        if ((e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess) return cuda_fail(e, "two-pass join");
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "FP32 two-pass launch");
    return HEART_OK;
}

namespace {
struct DeviceWave {
    std::mutex m;
    void *buf = nullptr;
    uint32_t cap = 0;
    cudaEvent_t done = nullptr;               // recorded after the queue's last user
    cudaStream_t side = nullptr;              // the second stream of the two-pass trace
    cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kMaxDevices = 64;
DeviceWave g_wave[kMaxDevices];
}  // namespace

static void wave_side(cudaStream_t *side, cudaEvent_t *fork, cudaEvent_t *join) {
    int dev = 0;
    *side = nullptr;
    *fork = *join = nullptr;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
    const DeviceWave &W = g_wave[dev];
    *side = W.side;
    *fork = W.fork;
    *join = W.join;
}

heart_status wave_acquire(uint64_t n, cudaStream_t st, WaveLease *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(HEART_EINVAL, "device index beyond the hit-queue table");
    DeviceWave &W = g_wave[dev];
    W.m.lock();
    if (!W.done && (e = cudaEventCreateWithFlags(&W.done, cudaEventDisableTiming)) != cudaSuccess) {
        W.done = nullptr;
        W.m.unlock();
        return cuda_fail(e, "cudaEventCreate hit queue");
    }
    const uint32_t cap = wave_cap_for(n);
    if (!W.buf || W.cap < cap) {
        // a larger chunk than before: the previous user must be done before the queue is replaced
        if ((e = cudaEventSynchronize(W.done)) != cudaSuccess) { W.m.unlock(); return cuda_fail(e, "hit queue"); }
        if (W.buf) cudaFree(W.buf);
        W.buf = nullptr;
        W.cap = 0;
        if ((e = cudaMalloc(&W.buf, wave_bytes(cap))) != cudaSuccess) {
            W.buf = nullptr;
            W.m.unlock();
            return cuda_fail(e, "cudaMalloc hit queue");
        }
        W.cap = cap;
    }
    if (!W.side) {
        // the side stream and its events (a failure leaves the trace on the caller's stream alone)
        if (cudaStreamCreateWithFlags(&W.side, cudaStreamNonBlocking) != cudaSuccess) W.side = nullptr;
        if (cudaEventCreateWithFlags(&W.fork, cudaEventDisableTiming) != cudaSuccess) W.fork = nullptr;
        if (cudaEventCreateWithFlags(&W.join, cudaEventDisableTiming) != cudaSuccess) W.join = nullptr;
        cudaGetLastError();
    }
    if ((e = cudaStreamWaitEvent(st, W.done, 0)) != cudaSuccess) { W.m.unlock(); return cuda_fail(e, "hit queue"); }
    out->buf = W.buf;
    out->cap = W.cap;
    out->device = dev;
    return HEART_OK;
}

void wave_release(const WaveLease &lease, cudaStream_t st) {
    DeviceWave &W = g_wave[lease.device];
    cudaEventRecord(W.done, st);
    W.m.unlock();
}

heart_status launch_fp32(const SpecParams &S, const SourceParams &P, uint64_t n, uint64_t seed, uint64_t offset,
                         void *img, unsigned long long *scratch, cudaStream_t st, const QeParams *qe, void *wave,
                         uint32_t wave_cap, heart_ray_record *rec) {
    if (!wave || n == 0 || !takes_two_pass(S, P))
        return launch_single(S, P, n, seed, offset, img, scratch, rec, st, qe);
    // the two-pass trace: the per-ray work in its own pass, then the walk
    Launch32 L;
    make_launch32(S, P, n, seed, offset, L);
    L.img = img;
    L.tally = scratch;
    L.rec = rec;
    if (qe) {
        L.eimg = qe->eimg;
        L.n_qe = qe->n;
        for (int i = 0; i < qe->n; ++i) { L.qe_e[i] = (float)qe->keV[i]; L.qe_v[i] = (float)qe->qe[i]; }
    }
    WaveBuf B;
    B.base = wave;
    B.cap = wave_cap;
    B.pad = 0;
    unsigned long long *ctr = (unsigned long long *)((char *)wave + 2 * wave_buffer_bytes(wave_cap));
    if (rec) {
        // per-ray records (tests): the variant that carries p and dispatches the rocking
        // curve at run time, with the record writes; it runs the same device functions
        // as the variants below, so every ray takes the same decisions
        const bool F = L.geometry == HEART_FLAT;
        if (P.user) return F ? launch_wave_t<HEART_FLAT, -1, true, true, false, true>(L, B, n, ctr, st)
                             : launch_wave_t<HEART_CYL_VON_HAMOS, -1, true, true, false, true>(L, B, n, ctr, st);
        if (S.n_orders > 1) return F ? launch_wave_t<HEART_FLAT, -1, true, false, true, true>(L, B, n, ctr, st)
                                     : launch_wave_t<HEART_CYL_VON_HAMOS, -1, true, false, true, true>(L, B, n, ctr, st);
        return F ? launch_wave_t<HEART_FLAT, -1, true, false, false, true>(L, B, n, ctr, st)
                 : launch_wave_t<HEART_CYL_VON_HAMOS, -1, true, false, false, true>(L, B, n, ctr, st);
    }
    if (P.user) {
        // user-supplied rays (polarised or not): entered in FP64 by the spawn pass,
        // walked by the variant that carries p
        if (L.geometry == HEART_FLAT) return launch_wave_t<HEART_FLAT, -1, true, true>(L, B, n, ctr, st);
        return launch_wave_t<HEART_CYL_VON_HAMOS, -1, true, true>(L, B, n, ctr, st);
    }
    if (S.n_orders > 1) {
        // several orders: the polarised variant (run-time rocking curve) with per-order lane state
        if (L.geometry == HEART_FLAT) return launch_wave_t<HEART_FLAT, -1, true, false, true>(L, B, n, ctr, st);
        return launch_wave_t<HEART_CYL_VON_HAMOS, -1, true, false, true>(L, B, n, ctr, st);
    }
    if (P.pol_on || S.irc == HEART_IRC_NONE) {
        // polarised source: 112-byte records and the walk variant that carries p,
        // with the rocking curve dispatched at run time (one instantiation per
        // geometry); the walk without rocking curve (cone candidates) runs there too
        if (L.geometry == HEART_FLAT) return launch_wave_t<HEART_FLAT, -1, true>(L, B, n, ctr, st);
        return launch_wave_t<HEART_CYL_VON_HAMOS, -1, true>(L, B, n, ctr, st);
    }
#define HEART_WAVE_CASES(G)                                                                          \
    switch (L.irc_kind) {                                                                            \
    case HEART_IRC_DARWIN: return launch_wave_t<G, HEART_IRC_DARWIN>(L, B, n, ctr, st);             \
    case HEART_IRC_DARWIN_PRINS: return launch_wave_t<G, HEART_IRC_DARWIN_PRINS>(L, B, n, ctr, st); \
    case HEART_IRC_PSEUDO_VOIGT: return launch_wave_t<G, HEART_IRC_PSEUDO_VOIGT>(L, B, n, ctr, st); \
    case HEART_IRC_GAUSSIAN: return launch_wave_t<G, HEART_IRC_GAUSSIAN>(L, B, n, ctr, st);         \
    case HEART_IRC_LORENTZIAN: return launch_wave_t<G, HEART_IRC_LORENTZIAN>(L, B, n, ctr, st);     \
    default: return launch_wave_t<G, HEART_IRC_BOX>(L, B, n, ctr, st);                               \
    }
    if (L.geometry == HEART_FLAT) { HEART_WAVE_CASES(HEART_FLAT) } else { HEART_WAVE_CASES(HEART_CYL_VON_HAMOS) }
#undef HEART_WAVE_CASES
}

heart_status launch_fp32_records(const SpecParams &S, const SourceParams &P, uint64_t n, uint64_t seed,
                                 uint64_t offset, void *img, unsigned long long *scratch, heart_ray_record *rec,
                                 cudaStream_t st, const QeParams *qe) {
    return launch_single(S, P, n, seed, offset, img, scratch, rec, st, qe);
}

// Device block of a batched launch:
// [Launch32 x n][chunk_begin x (n + 1)][tallies x n x kTallyN][counter]
size_t batch_bytes(int n) {
    size_t a = (size_t)n * sizeof(Launch32);
    a = (a + 15) & ~(size_t)15;
    a += (size_t)(n + 1) * 8;
    a = (a + 15) & ~(size_t)15;
    a += (size_t)n * kTallyN * 8 + 16;
    return a;
}

size_t spectra_bytes(const std::vector<unsigned char> *spectra, int n) {
    size_t a = 0;
    for (int i = 0; spectra && i < n; ++i) a += (spectra[i].size() + 15) & ~(size_t)15;
    return a;
}

heart_status launch_batch(const SpecParams *const *S, const SourceParams *P, const uint64_t *n_rays,
                          const uint64_t *seeds, const uint64_t *offsets, void *const *imgs, int n, void *dev,
                          std::vector<unsigned char> &host, cudaStream_t st, unsigned long long **tallies_dev,
                          unsigned long long *const *tally_ptrs, const std::vector<unsigned char> *spectra,
                          unsigned char *pinned, size_t pinned_cap) {
    const size_t base = batch_bytes(n);
    const size_t total = base + spectra_bytes(spectra, n);
    // the host image of the block: in the caller's pinned buffer when it is large enough
    // (an asynchronous upload), else in `host` (pageable: staged before the copy returns)
    unsigned char *hb;
    if (pinned && pinned_cap >= total) {
        hb = pinned;
        std::memset(hb, 0, total);
    } else {
        host.assign(total, 0);
        hb = host.data();
    }
    Launch32 *jobs = (Launch32 *)hb;
    const size_t off_cb = ((size_t)n * sizeof(Launch32) + 15) & ~(size_t)15;
    const size_t off_t = (off_cb + (size_t)(n + 1) * 8 + 15) & ~(size_t)15;
    const size_t off_c = off_t + (size_t)n * kTallyN * 8;
    unsigned long long *cb = (unsigned long long *)(hb + off_cb);
    unsigned char *d = (unsigned char *)dev;
    uint64_t all_rays = 0;
    bool ext = false;
    for (int i = 0; i < n; ++i) {
        all_rays += n_rays[i];
        ext |= P[i].pol_on || P[i].user || S[i]->n_orders > 1;
    }
    const uint32_t chunk = chunk_for(all_rays);
    unsigned long long nch = 0;
    size_t sp_off = base;
    for (int i = 0; i < n; ++i) {
        SourceParams Pi = P[i];
        if (spectra && !spectra[i].empty()) {
            // the job's tabulated spectrum rides after the work plan
            std::memcpy(hb + sp_off, spectra[i].data(), spectra[i].size());
            bind_spectrum(&Pi, d + sp_off);
            sp_off += (spectra[i].size() + 15) & ~(size_t)15;
        }
        make_launch32(*S[i], Pi, n_rays[i], seeds[i], offsets ? offsets[i] : 0, jobs[i]);
        jobs[i].img = imgs[i];
        jobs[i].tally = tally_ptrs ? tally_ptrs[i] : (unsigned long long *)(d + off_t) + (size_t)i * kTallyN;
        jobs[i].rec = nullptr;
        cb[i] = nch;
        nch += (n_rays[i] + chunk - 1) / chunk;
    }
    cb[n] = nch;
    *tallies_dev = (unsigned long long *)(d + off_t);
    cudaError_t e = cudaMemcpyAsync(dev, hb, total, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch upload");
    if (nch == 0) return HEART_OK;
    WorkPlan W;
    std::memset(&W, 0, sizeof W);
    W.jobs = (const Launch32 *)d;
    W.chunk_begin = (const unsigned long long *)(d + off_cb);
    W.n_jobs = n;
    W.chunk_rays = chunk;
    W.n_chunks = nch;
    W.counter = (unsigned long long *)(d + off_c);
    Launch32 dummy;
    std::memset(&dummy, 0, sizeof dummy);
    return dispatch<false>(dummy, W, st, true, ext);
}

}  // namespace heart

extern "C" heart_status heart_trace_batch(heart_spectrometer *const *specs, const heart_source_desc *const *srcs,
                                          const uint64_t *n_rays, const uint64_t *seeds, void *const *d_images,
                                          int32_t n_jobs, void *stream, heart_tally *out) {
    using namespace heart;
    if (n_jobs == 0) return HEART_OK;
    if (n_jobs < 0 || !specs || !srcs || !n_rays || !seeds || !d_images) return fail(HEART_EINVAL, "null batch array");
    std::vector<SourceParams> P((size_t)n_jobs);
    std::vector<std::vector<unsigned char>> spectra((size_t)n_jobs);
    std::vector<const SpecParams *> S((size_t)n_jobs);
    char err[256] = {0};
    for (int i = 0; i < n_jobs; ++i) {
        if (!specs[i]) return fail(HEART_EINVAL, "null spectrometer in batch");
        const size_t elt = specs[i]->p.count_type == HEART_COUNT_I64 ? 8 : 4;
        if (!d_images[i] || ((uintptr_t)d_images[i] % elt) != 0) return fail(HEART_EINVAL, "null or misaligned image in batch");
        heart_status st = build_source_params(srcs[i], &P[i], err, (int)sizeof err, &spectra[i]);
        if (st != HEART_OK) return fail(st, err);
        S[i] = &specs[i]->p;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    // Jobs of kTwoPassMinRays rays or more that the two-pass trace takes (one
    // reflection order) run as single-job two-pass launches, as single traces and
    // the request loop run them; the others share one persistent launch.
    std::vector<int> big, small;
    for (int i = 0; i < n_jobs; ++i)
        (n_rays[i] >= kTwoPassMinRays && takes_two_pass(*S[i], P[i]) ? big : small).push_back(i);
    // device block: [tallies x n_jobs][big jobs' spectra][the persistent launch's block]
    const size_t tall_bytes = ((size_t)n_jobs * kTallyN * 8 + 15) & ~(size_t)15;
    size_t big_sp = 0;
    uint64_t big_max = 0;
    for (int i : big) {
        big_sp += (spectra[i].size() + 15) & ~(size_t)15;
        big_max = n_rays[i] > big_max ? n_rays[i] : big_max;
    }
    const int ns = (int)small.size();
    std::vector<const SpecParams *> sS;
    std::vector<SourceParams> sP;
    std::vector<std::vector<unsigned char>> sSp;
    std::vector<uint64_t> sN, sSeed;
    std::vector<void *> sImg;
    for (int i : small) {
        sS.push_back(S[i]); sP.push_back(P[i]); sSp.push_back(spectra[i]);
        sN.push_back(n_rays[i]); sSeed.push_back(seeds[i]); sImg.push_back(d_images[i]);
    }
    const size_t bytes = tall_bytes + big_sp + (ns ? batch_bytes(ns) + spectra_bytes(sSp.data(), ns) : 0);
    unsigned char *dev = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&dev, bytes, cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync batch");
    unsigned long long *tall = (unsigned long long *)dev;
    heart_status st = HEART_OK;
    e = cudaMemsetAsync(tall, 0, tall_bytes, cs);
    if (e != cudaSuccess) st = cuda_fail(e, "batch tallies");
    if (st == HEART_OK && !big.empty()) {
        WaveLease lease{nullptr, 0u, 0};
        st = wave_acquire(big_max, cs, &lease);
        const bool held = st == HEART_OK;
        size_t off = tall_bytes;
        for (size_t b = 0; st == HEART_OK && b < big.size(); ++b) {
            const int i = big[b];
            SourceParams Pi = P[i];
            if (!spectra[i].empty()) {
                // pageable source: staged before the call returns
                e = cudaMemcpyAsync(dev + off, spectra[i].data(), spectra[i].size(), cudaMemcpyHostToDevice, cs);
                if (e != cudaSuccess) { st = cuda_fail(e, "spectrum upload"); break; }
                bind_spectrum(&Pi, dev + off);
                off += (spectra[i].size() + 15) & ~(size_t)15;
            }
            st = launch_fp32(*S[i], Pi, n_rays[i], seeds[i], 0, d_images[i], tall + (size_t)i * kTallyN, cs, nullptr,
                             lease.buf, lease.cap);
        }
        if (held) wave_release(lease, cs);
    }
    std::vector<unsigned char> host;
    if (st == HEART_OK && ns) {
        std::vector<unsigned long long *> tptr;
        for (int i : small) tptr.push_back(tall + (size_t)i * kTallyN);
        unsigned long long *unused = nullptr;
        st = launch_batch(sS.data(), sP.data(), sN.data(), sSeed.data(), nullptr, sImg.data(), ns,
                          dev + tall_bytes + big_sp, host, cs, &unused, tptr.data(), sSp.data());
    }
    if (st == HEART_OK && out) {
        std::vector<unsigned long long> h((size_t)n_jobs * kTallyN);
        e = cudaMemcpyAsync(h.data(), tall, h.size() * 8, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) st = cuda_fail(e, "batch tallies");
        bool stuck = false;
        for (int i = 0; st == HEART_OK && i < n_jobs; ++i) {
            std::memcpy(&out[i], &h[(size_t)i * kTallyN], sizeof(heart_tally));
            stuck |= out[i].stuck > 0;
        }
        if (st == HEART_OK && stuck) st = fail(HEART_ELIMIT, "a ray reached the collision cap");
    }
    cudaFreeAsync(dev, cs);
    return st;
}

// ---------------------------------------------------------------------------
// autotuner: time candidate launch shapes on a probe and keep the fastest
// ---------------------------------------------------------------------------
extern "C" heart_status heart_autotune(heart_spectrometer *h, const heart_source_desc *src, uint64_t probe_rays,
                                       void *stream, heart_tune *out) {
    using namespace heart;
    if (!h) return fail(HEART_EINVAL, "null spectrometer");
    if (probe_rays < 4096) return fail(HEART_EINVAL, "probe needs at least 4096 rays");
    SourceParams P;
    char err[256] = {0};
    std::vector<unsigned char> spectrum;
    heart_status st = build_source_params(src, &P, err, (int)sizeof err, &spectrum);
    if (st != HEART_OK) return fail(st, err);
    cudaStream_t cs = (cudaStream_t)stream;
    // the two-pass probes use the device's hit queue, held for the whole tuning
    const bool two_pass = takes_two_pass(h->p, P);
    WaveLease lease{nullptr, 0u, 0};
    if (two_pass) {
        st = wave_acquire(probe_rays, cs, &lease);
        if (st != HEART_OK) return st;
    }
    struct ReleaseOnExit {
        bool on;
        const WaveLease &l;
        cudaStream_t s;
        ~ReleaseOnExit() { if (on) wave_release(l, s); }
    } release_lease{two_pass, lease, cs};
    void *d_spec = nullptr;
    if (!spectrum.empty()) {
        cudaError_t e0 = cudaMallocAsync(&d_spec, spectrum.size(), cs);
        if (e0 == cudaSuccess) e0 = cudaMemcpyAsync(d_spec, spectrum.data(), spectrum.size(), cudaMemcpyHostToDevice, cs);
        if (e0 != cudaSuccess) {
            if (d_spec) cudaFreeAsync(d_spec, cs);
            return cuda_fail(e0, "spectrum upload");
        }
        bind_spectrum(&P, d_spec);
    }
    struct FreeOnExit {
        void *p;
        cudaStream_t s;
        ~FreeOnExit() { if (p) cudaFreeAsync(p, s); }
    } free_spec{d_spec, cs};
    const size_t elt = h->p.count_type == HEART_COUNT_I64 ? 8 : 4;
    const size_t bytes = (size_t)h->p.nx * h->p.ny * elt;
    cudaError_t e;
    if (!h->d_image_host_path || h->host_image_bytes < bytes) {
        if (h->d_image_host_path) cudaFree(h->d_image_host_path);
        h->d_image_host_path = nullptr;
        if ((e = cudaMalloc(&h->d_image_host_path, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc image");
        h->host_image_bytes = bytes;
    }
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    // Two knots, each timed on the kernel it shapes: the refill threshold on this
    // trace's own path (the two-pass trace when it applies), then the persistent
    // kernel's blocks per SM (batched and served jobs, records of user rays with
    // several orders) on that kernel with the chosen threshold.  A probe is timed
    // after one warm-up run.
    const TuneConfig saved = g_tune;
    auto probe = [&](bool persistent, double &rate) -> heart_status {
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaMemsetAsync(h->d_scratch, 0, kScratchWords * sizeof(unsigned long long), cs);
            cudaEventRecord(t0, cs);
            heart_status s2 = launch_fp32(h->p, P, probe_rays, 0x5eed + rep, 0, h->d_image_host_path, h->d_scratch,
                                          cs, nullptr, persistent ? nullptr : lease.buf, lease.cap);
            cudaEventRecord(t1, cs);
            if (s2 != HEART_OK) return s2;
            if ((e = cudaEventSynchronize(t1)) != cudaSuccess) return cuda_fail(e, "autotune probe");
            cudaEventElapsedTime(&ms, t0, t1);
        }
        rate = (double)probe_rays / (ms * 1e-3);
        return HEART_OK;
    };
    const int refills[4] = {1, 4, 8, 16};
    const int occs[2] = {6, 5};
    TuneConfig best = g_tune;
    double best_rate = -1.0, rate = 0.0;
    for (int ri = 0; ri < 4 && st == HEART_OK; ++ri) {
        g_tune.refill = refills[ri];
        st = probe(!two_pass, rate);
        if (st == HEART_OK && rate > best_rate) { best_rate = rate; best.refill = refills[ri]; }
    }
    g_tune.refill = best.refill;
    double best_occ_rate = -1.0;
    for (int oi = 0; oi < 2 && st == HEART_OK; ++oi) {
        g_tune.blocks_per_sm = occs[oi];
        st = probe(true, rate);
        if (st == HEART_OK && rate > best_occ_rate) { best_occ_rate = rate; best.blocks_per_sm = occs[oi]; }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st != HEART_OK) { g_tune = saved; return st; }
    g_tune = best;
    if (out) {
        out->blocks_per_sm = best.blocks_per_sm;
        out->refill_lanes = best.refill;
        out->max_chunk_rays = best.chunk_rays;
        out->reserved = 0;
        out->rays_per_s = best_rate;
    }
    return HEART_OK;
}

// ---------------------------------------------------------------------------
// Batched trace without any allocation.
//
// Some callers cannot allocate device memory while they run: an application
// that hands all free device memory to its own pool at start-up, or a
// control loop that must never risk an allocation failure or the implicit
// synchronisation an allocation can cause.  heart_trace_batch needs a small
// per-call work area (job table, work counter, tallies) and allocates it on
// the stream; this variant runs the same batched kernel on a work area that
// lives in a fixed, file-scope device array instead, so a call allocates
// nothing on the device.  The array holds at most kStaticMaxJobs jobs, every
// GPU that loads the library keeps it until the process exits, and all calls
// share it: each call rewrites it completely (work counter and tallies start
// at zero), and calls that overlap on the GPU race on it.
// ---------------------------------------------------------------------------
namespace heart {
namespace {

constexpr int kStaticMaxJobs = HEART_STATIC_MAX_JOBS;
constexpr size_t kStaticJobsBytes = ((size_t)kStaticMaxJobs * sizeof(Launch32) + 15) & ~(size_t)15;
constexpr size_t kStaticChunkBytes = (((size_t)kStaticMaxJobs + 1) * 8 + 15) & ~(size_t)15;
constexpr size_t kStaticTallyBytes = (size_t)kStaticMaxJobs * kTallyN * 8;
constexpr size_t kStaticBytes = kStaticJobsBytes + kStaticChunkBytes + kStaticTallyBytes + 16;

static __device__ __align__(256) unsigned char g_static_work[kStaticBytes];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;                                 // serialises the host staging below
void *g_static_dev[kStaticMaxDevices] = {nullptr};      // device address of g_static_work, per device
unsigned char g_static_host[kStaticBytes];              // host image of the work area
SourceParams g_static_src[kStaticMaxJobs];

}  // namespace
}  // namespace heart

extern "C" heart_status heart_trace_batch_static(heart_spectrometer *const *specs,
                                                 const heart_source_desc *const *srcs, const uint64_t *n_rays,
                                                 const uint64_t *seeds, void *const *d_images, int32_t n_jobs,
                                                 void *stream, heart_tally *out) {
    using namespace heart;
    if (n_jobs == 0) return HEART_OK;
    if (n_jobs < 0) return fail(HEART_EINVAL, "negative job count");
    if (n_jobs > kStaticMaxJobs)
        return fail(HEART_EINVAL, "heart_trace_batch_static: more jobs than HEART_STATIC_MAX_JOBS (64)");
    if (!specs || !srcs || !n_rays || !seeds || !d_images) return fail(HEART_EINVAL, "null batch array");
    std::lock_guard<std::mutex> lk(g_static_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kStaticMaxDevices) return fail(HEART_EINVAL, "device ordinal out of range");
    if (!g_static_dev[dev]) {
        // once per device, with that device current: the array's device address
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_work);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        g_static_dev[dev] = ptr;
    }
    unsigned char *d = (unsigned char *)g_static_dev[dev];
    char err[256] = {0};
    for (int i = 0; i < n_jobs; ++i) {
        if (!specs[i]) return fail(HEART_EINVAL, "null spectrometer in batch");
        const size_t elt = specs[i]->p.count_type == HEART_COUNT_I64 ? 8 : 4;
        if (!d_images[i] || ((uintptr_t)d_images[i] % elt) != 0) return fail(HEART_EINVAL, "null or misaligned image in batch");
        heart_status st = build_source_params(srcs[i], &g_static_src[i], err, (int)sizeof err);
        if (st != HEART_OK) return fail(st, err);
    }
    // host image of the work area: job table, chunk table, zero tallies and counter
    std::memset(g_static_host, 0, kStaticBytes);
    Launch32 *jobs = (Launch32 *)g_static_host;
    unsigned long long *cb = (unsigned long long *)(g_static_host + kStaticJobsBytes);
    unsigned long long *d_tallies = (unsigned long long *)(d + kStaticJobsBytes + kStaticChunkBytes);
    // work items sized to the whole batch, as heart_trace_batch sizes them, so that a
    // batch of small jobs still spreads over the SMs
    uint64_t total = 0;
    for (int i = 0; i < n_jobs; ++i) total += n_rays[i];
    const uint32_t chunk = chunk_for(total);
    unsigned long long nch = 0;
    bool ext = false;
    for (int i = 0; i < n_jobs; ++i) {
        ext |= g_static_src[i].pol_on != 0 || specs[i]->p.n_orders > 1;
        make_launch32(specs[i]->p, g_static_src[i], n_rays[i], seeds[i], 0, jobs[i]);
        jobs[i].img = d_images[i];
        jobs[i].tally = d_tallies + (size_t)i * kTallyN;
        jobs[i].rec = nullptr;
        cb[i] = nch;
        nch += (n_rays[i] + chunk - 1) / chunk;
    }
    cb[n_jobs] = nch;
    cudaStream_t cs = (cudaStream_t)stream;
    // pageable source: staged before the call returns, so the buffer can be reused
    e = cudaMemcpyAsync(d, g_static_host, kStaticBytes, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "work area upload");
    if (nch > 0) {
        WorkPlan W;
        std::memset(&W, 0, sizeof W);
        W.jobs = (const Launch32 *)d;
        W.chunk_begin = (const unsigned long long *)(d + kStaticJobsBytes);
        W.n_jobs = n_jobs;
        W.chunk_rays = chunk;
        W.n_chunks = nch;
        W.counter = (unsigned long long *)(d + kStaticJobsBytes + kStaticChunkBytes + kStaticTallyBytes);
        Launch32 dummy;
        std::memset(&dummy, 0, sizeof dummy);
        heart_status st = dispatch<false>(dummy, W, cs, true, ext);
        if (st != HEART_OK) return st;
    }
    if (out) {
        unsigned long long *h = (unsigned long long *)(g_static_host + kStaticJobsBytes + kStaticChunkBytes);
        e = cudaMemcpyAsync(h, d_tallies, (size_t)n_jobs * kTallyN * 8, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) return cuda_fail(e, "tally read-back");
        bool stuck = false;
        for (int i = 0; i < n_jobs; ++i) {
            std::memcpy(&out[i], h + (size_t)i * kTallyN, sizeof(heart_tally));
            stuck |= out[i].stuck > 0;
        }
        if (stuck) return fail(HEART_ELIMIT, "a ray reached the collision cap");
    }
    return HEART_OK;
}

// ---------------------------------------------------------------------------
// test support: device functions on arrays
// ---------------------------------------------------------------------------
extern "C" heart_status heart_check_functions(heart_spectrometer *h, int32_t which, const float *d_x,
                                              const float *d_y, const float *d_z, float *d_out, uint64_t n,
                                              void *stream) {
    using namespace heart;
    if (which < 0 || which > 4) return fail(HEART_EINVAL, "unknown function");
    if (!d_x || !d_out || ((which == 0 || which >= 3) && !d_y) || (which >= 3 && !d_z))
        return fail(HEART_EINVAL, "null array");
    if ((which == 1 || which == 2) && !h) return fail(HEART_EINVAL, "null spectrometer");
    if (n == 0) return HEART_OK;
    Launch32 L;
    std::memset(&L, 0, sizeof L);
    if (h) {
        // the spectrometer's rocking-curve constants (a monochromatic point source fills the rest)
        heart_spectral_component c;
        std::memset(&c, 0, sizeof c);
        c.kind = HEART_SRC_MONO;
        c.e0_keV = 8.0;
        c.weight = 1.0;
        heart_source_desc d;
        std::memset(&d, 0, sizeof d);
        d.components = &c;
        d.n_components = 1;
        d.axis[0] = 1.0;
        SourceParams P;
        char err[256] = {0};
        heart_status st = build_source_params(&d, &P, err, (int)sizeof err);
        if (st != HEART_OK) return fail(st, err);
        make_launch32(h->p, P, n, 1, 0, L);
    }
    const int blocks = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)num_sms() * 8);
    k_check_functions<<<blocks, 256, 0, (cudaStream_t)stream>>>(L, which, d_x, d_y, d_z, d_out, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "check kernel");
    return HEART_OK;
}
