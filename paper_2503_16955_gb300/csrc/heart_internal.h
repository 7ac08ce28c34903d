// heart_internal.h -- parameter blocks shared by the host set-up code and the
// CUDA kernels of the library (not part of the public ABI).
#pragma once
#include <stdint.h>

#include "heart.h"

namespace heart {

constexpr int kMdfM = 4096;      // body knots of the mosaic inverse CDF, u = i / 4096
constexpr int kMdfT = 256;       // tail intervals, linear in tau = -log2(1 - u), tau in [12, 33]
constexpr int kMdfKnots = kMdfM + kMdfT + 1;
constexpr int kMaxComp = 16;
constexpr int kTallyN = 27;      // heart_tally as 27 uint64 words

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
    // device tables: q = 1 - cos(theta) at the body knots then the tail knots
    const double *mdf64;
    const float *mdf32;
};

struct SourceParams {
    int32_t n_comp, pad;
    int32_t kind[kMaxComp];
    double e0[kMaxComp], width[kMaxComp], lo[kMaxComp], hi[kMaxComp], cumw[kMaxComp];
    double lorentz_F0[kMaxComp];     // CDF of the untruncated Cauchy at E = 0
    double origin[3], ax[3], b1[3], b2[3];
    double one_minus_cos_max;        // 2 sin^2(cone / 2)
    double sig1, sig2;               // spot sigmas
};

// host set-up (heart_host.cpp)
heart_status build_spec_params(const heart_spectrometer_desc *d, SpecParams *p, double *mdf_table,
                               char *err, int errlen);
heart_status build_source_params(const heart_source_desc *s, SourceParams *p, char *err, int errlen);

}  // namespace heart
