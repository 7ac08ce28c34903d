// heart_internal.h -- parameter blocks shared by the host set-up code and the
// CUDA kernels of the library (not part of the public ABI).
#pragma once
#include <stdint.h>

#include <vector>

#include "heart.h"

namespace heart {

constexpr int kMdfM = 4096;      // body knots of the mosaic inverse CDF, u = i / 4096
constexpr int kMdfT = 256;       // tail intervals, linear in tau = -log2(1 - u), tau in [12, 33]
constexpr int kMdfKnots = kMdfM + kMdfT + 1;
constexpr int kMaxComp = 16;
constexpr int kMaxQe = 32;       // detector quantum-efficiency knots
constexpr int kTallyN = 27;      // heart_tally as 27 uint64 words
constexpr int kMaxTable = HEART_MAX_TABLE;   // knots of a tabulated spectrum
// thinned sampler: tilt-bound grid q_j = 2^(j/8 - 48), j < kQGrid, with the
// first mosaic-table word of the interval holding each q_j
constexpr int kQGrid = 392;
// process (b) of one reflection order splits into band B, the grid points from
// kBandDJ steps above q_min's (a factor 2^1.5 in q) to kBandJ2 (q = 2^(-33/8),
// theta = 0.34 rad), generated at its own arc-measure bound, and band A, the rest
constexpr int kBandDJ = 12, kBandJ2 = 351;

// tally word indices (same order as heart_tally)
enum : int {
    T_EMITTED = 0, T_MISS, T_ABSORBED, T_EXIT_FRONT, T_EXIT_BACK, T_EXIT_SIDE, T_CAPPED, T_STUCK,
    T_NO_BRAGG, T_DET_HITS, T_HIST0, T_COLLISIONS = T_HIST0 + 16
};

// Everything a kernel needs to trace one spectrometer, passed by value.
struct SpecParams {
    int32_t geometry, irc, max_refl, count_type;
    int64_t max_coll;
    double thickness, radius;
    double c[3];                     // flat: front-face centre; cylinder: point on the axis
    double N[3], ed[3], en[3];       // flat frame: normal, dispersive, non-dispersive
    double ax[3], cc[3], ww[3];      // cylinder frame: axis, centre direction, ax x cc
    double zc;                       // cylinder: axial coordinate of the crystal centre
    double half_d, half_n;           // flat: half extents; cylinder: half axial length, unused
    double sphi, cphi;               // cylinder: sin / cos of the half arc angle
    // intrinsic rocking curve, argument x = Delta - Delta_M
    double irc_fwhm, irc_eta, irc_delta, irc_norm, irc_g, irc_shift, irc_max;
    // per-energy physics
    double d_A, labs, labs_ref, labs_pow, K;
    // detector
    double D0[3], eu[3], ev[3], nd[3];
    int32_t nx, ny;
    double pix;
    // candidate sampler: thinned (0) or plain (1); v* and the IRC half-width X*
    // beyond which R / R_max <= v*
    int32_t sampler, pad_s;
    double vstar, xstar;
    // reflection orders (n_orders >= 1): multiple, K ratio, width ratio
    int32_t n_orders, n_irc_e;
    int32_t ord_m[HEART_MAX_ORDERS];
    double ord_k[HEART_MAX_ORDERS], ord_w[HEART_MAX_ORDERS];
    // energy-dependent rocking curve: knots, width scale, added shift
    double irc_e[HEART_MAX_IRC_E], irc_ws[HEART_MAX_IRC_E], irc_sh[HEART_MAX_IRC_E];
    // no rocking curve: the cone-candidate rate factor 2 W(0) / int W dq, and
    // the mosaic distribution's W(q) / W(0) in closed form (mdf_ratio): theta
    // shapes w_wl a2 / (a2 + theta^2) + w_wg exp(-w_c theta^2); vMF
    // exp(-w_c q); WL a2 / (a2 + 2 q); SWL w_b^2 / (w_b + q)^2; uniform q <= w_qmax
    int32_t mdf, pad_m;
    double none_fac, w_a2, w_c, w_wl, w_wg, w_b, w_qmax;
    // no rocking curve, thinned: a tilt q_v with W(q) / W(0) <= v* for q >= q_v (infinite if none)
    double none_qv;
    // device tables: q = 1 - cos(theta) at the body knots then the tail knots
    const double *mdf64;
    const float *mdf32;
    const uint32_t *qgrid;           // kQGrid words (thinned sampler)
    uint32_t band_w2, pad_b;         // qgrid[kBandJ2]: the first table word past band B
    // per grid point j: 1 / sin(theta) at the table knot that starts qgrid[j]'s interval
    // (rounded up; 0 where the knot is 0): band B's smallest tilt when it starts at j
    const float *band_is1;
};

struct SourceParams {
    int32_t n_comp, pad;
    int32_t kind[kMaxComp];
    double e0[kMaxComp], width[kMaxComp], lo[kMaxComp], hi[kMaxComp], cumw[kMaxComp];
    double lorentz_F0[kMaxComp];     // CDF of the untruncated Cauchy at E = 0
    double origin[3], ax[3], b1[3], b2[3];
    double one_minus_cos_max;        // 2 sin^2(cone / 2)
    double sig1, sig2;               // spot sigmas
    double pol[3];                   // linear polarisation (unit), if pol_on
    int32_t pol_on, user;            // polarised source; rays come from user arrays
    const double *ray[10];           // user arrays: ox oy oz kx ky kz E px py pz (p* may be null)
    // tabulated spectrum (device copy, see bind_spectrum): CDF and energies at
    // the knots for the FP64 path; for the FP32 path the CDF as thresholds on
    // the raw 32-bit word, the in-interval offsets and slopes, and the knots
    // relative to the table's mean energy
    int32_t n_tab, pad_tab;
    double tab_mean;
    const double *tab_cdf, *tab_keV;
    const unsigned long long *tab_thr;
    const float *tab_off, *tab_inv, *tab_dE, *tab_w;
};

// device image of a tabulated spectrum of n knots (bind_spectrum's layout)
inline size_t spectrum_bytes(int n) { return (size_t)n * 40; }
// point the table fields of p at a device copy of the host image
inline void bind_spectrum(SourceParams *p, const void *dev) {
    const unsigned char *d = (const unsigned char *)dev;
    const size_t n = (size_t)p->n_tab;
    p->tab_cdf = (const double *)d;
    p->tab_keV = (const double *)(d + 8 * n);
    p->tab_thr = (const unsigned long long *)(d + 16 * n);
    p->tab_off = (const float *)(d + 24 * n);
    p->tab_inv = (const float *)(d + 28 * n);
    p->tab_dE = (const float *)(d + 32 * n);
    p->tab_w = (const float *)(d + 36 * n);
}

// optional energy image: each detected photon adds round(E * QE(E) * 1e6)
// (units of 1e-6 keV) to eimg; QE linear between knots, clamped beyond
struct QeParams {
    int32_t n, pad;
    double keV[kMaxQe], qe[kMaxQe];
    unsigned long long *eimg;
};

// host set-up (heart_host.cpp)
heart_status build_spec_params(const heart_spectrometer_desc *d, SpecParams *p, double *mdf_table,
                               char *err, int errlen);
// spectrum: host image of the source's tabulated spectrum when a component
// uses it (then bind_spectrum after the upload); nullptr: tables rejected
heart_status build_source_params(const heart_source_desc *s, SourceParams *p, char *err, int errlen,
                                 std::vector<unsigned char> *spectrum = nullptr);
heart_status build_ray_params(const heart_ray_arrays *r, SourceParams *p, char *err, int errlen);
heart_status build_qe_params(const heart_qe_table *q, unsigned long long *eimg, QeParams *p, char *err, int errlen);

}  // namespace heart
