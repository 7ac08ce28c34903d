/*
 * heart_oracle.h -- plain FP64 CPU oracle of the mosaic-crystal ray path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the package, its CUDA
 * kernels, its C-ABI library) includes, links or calls this code.  Only the
 * tests, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm
 * load liboracle.so.  The oracle shares no header, helper, table generator or
 * constant with the GPU path; the two agree only through the written
 * specification of the sampling model (Section 2 of the paper, restated in the
 * header comment of oracle.c).
 *
 * Every routine is the slow, obviously-correct form: positions in the global
 * frame, libm transcendental functions, adaptive Simpson quadrature, no
 * blocking or reordering beyond the paper's algorithm.
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   orc_philox4x32_10        pinned (PyTorch's Philox engine on matched key/counter)
 *   orc_pv_width             pinned (54.3 and 110.8 urad printed in Sec. 4.2)
 *   orc_irc                  pinned (unit area; Darwin 8/3 integral; DP -> Darwin as g -> 0)
 *   orc_mdf_*                pinned (closed-form quantiles of vMF, WL, SWL, uniform; sphere norms)
 *   orc_trace                pinned (Beer-Lambert, reflection rate vs quadrature of Eq. ReflXsection,
 *                                    von Hamos focus 2R cot(aB), conservation, thread invariance,
 *                                    hand-traced injected-uniform walks)
 *   orc_reflection_rate      pinned (small-Gamma limit Eq. SimpleZachXsection for vMF)
 *   orc_sample_crystallites  pinned (accepted Delta ~ IRC; psi ~ W(theta(psi)), Appendix Method II)
 *   polarised walk (G_pol, p update) pinned (sigma: G = 1, pi: G = cos^2 2a on hand-traced rays; the
 *                                    thresholds of two orthogonal p sum to twice the unpolarised one;
 *                                    closed-form reflected p; p stays unit and perpendicular to k)
 *   orc_trace_rays           pinned (rays repeating a zero-cone source reproduce orc_trace exactly)
 *   thinned sampler          pinned (near-Bragg segments replay the plain walk word for word;
 *                                    two-sample agreement with the plain walk on fans of directions for
 *                                    all 7 MDFs and 6 IRCs and on the workloads; first-reflection
 *                                    probability vs quadrature of Eq. ReflXsection)
 *   reflection orders        pinned (explicit first order = single reflection word for word; order m on d =
 *                                    order 1 on d/m; thin-slab reflection probability and per-order
 *                                    shares vs the quadrature summed over orders)
 *   energy-dependent IRC     pinned (constant table = wider, shifted curve; interpolation and clamping)
 *   IRC "none" (Bragg cone)  pinned (k_in . k_out = cos 2a~0 on every single reflection; thin-slab reflection
 *                                    probability vs quadrature along the cone and, for vMF, the Bessel closed
 *                                    form; the limit of ever narrower box curves; both samplers: the plain
 *                                    bound f(0) and the per-segment cone bounds agree)
 *   tabulated spectrum       pinned (KS against the piecewise-linear CDF written from the knots; a
 *                                    two-knot table reproduces the uniform component bit for bit)
 *   orc_trace_energy         pinned (mono line: energy image = E x QE x counts; QE interpolation)
 *   absolute reflectivity / detector image shapes against experiment: parity unpinned
 *   (the paper's measured spectra are not available).
 */
#ifndef HEART_ORACLE_H
#define HEART_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* geometry, mosaic distribution (MDF), intrinsic rocking curve (IRC) and
 * spectral-component codes: the numbering is part of the written interface
 * convention shared with the product by specification only. */
enum { ORC_FLAT = 0, ORC_CYL = 1 };
enum { ORC_MDF_GAUSSIAN = 0, ORC_MDF_LORENTZIAN = 1, ORC_MDF_PSEUDO_VOIGT = 2,
       ORC_MDF_VMF = 3, ORC_MDF_WL = 4, ORC_MDF_SWL = 5, ORC_MDF_UNIFORM = 6 };
enum { ORC_IRC_DARWIN = 0, ORC_IRC_DARWIN_PRINS = 1, ORC_IRC_PSEUDO_VOIGT = 2,
       ORC_IRC_GAUSSIAN = 3, ORC_IRC_LORENTZIAN = 4, ORC_IRC_BOX = 5,
       /* no rocking curve (Sec. 2.2.1, "none"): R(Delta) = delta(Delta), unit
        * area; crystallites reflect only at a~ = aB + Delta_M exactly */
       ORC_IRC_NONE = 6 };
enum { ORC_SRC_MONO = 0, ORC_SRC_GAUSS = 1, ORC_SRC_LORENTZ = 2, ORC_SRC_INV_E = 3,
       ORC_SRC_UNIFORM = 4, ORC_SRC_TABLE = 5 };
enum { ORC_MISS = 0, ORC_ABSORBED = 1, ORC_EXIT_FRONT = 2, ORC_EXIT_BACK = 3,
       ORC_EXIT_SIDE = 4, ORC_CAPPED = 5, ORC_STUCK = 6 };

#define ORC_MDF_M 4096        /* body quantile knots, uniform in u          */
#define ORC_MDF_T 256         /* tail intervals, uniform in -log2(1-u)      */
#define ORC_MAX_COMP 16
#define ORC_MAX_TABLE 8192    /* knots of a tabulated spectrum            */
#define ORC_MAX_ORDERS 4      /* reflection orders summed in the walk      */
#define ORC_MAX_IRC_E 16      /* knots of the energy-dependent IRC        */

typedef struct {
    double d_spacing_A;       /* d_H of Eq. BraggLaw, Angstrom */
    double thickness_mm;
    int32_t geometry;         /* ORC_FLAT / ORC_CYL */
    int32_t mdf;
    double radius_mm;         /* cylinder: radius of the reflecting (inner) face */
    double centre[3];         /* flat: centre of front face; cyl: point on the axis */
    double normal[3];         /* flat: front-face normal N; cyl: direction axis -> crystal centre */
    double axis[3];           /* flat: dispersive in-plane direction; cyl: cylinder axis */
    double centre_axial_mm;   /* cyl: axial coordinate of the crystal centre */
    double size_disp_mm;      /* flat: extent along axis; cyl: axial length */
    double size_nondisp_mm;   /* flat: extent along N x axis; cyl: arc length on r = R */
    double mdf_fwhm_rad;      /* Gamma */
    double mdf_eta;           /* pseudo-Voigt Lorentzian fraction */
    int32_t irc;
    int32_t max_reflections;
    double irc_fwhm_rad;      /* Darwin / DP: Darwin (g=0) FWHM; G, L, box: FWHM; pV: Gaussian FWHM */
    double irc_lorentz_fwhm_rad;  /* pV: Lorentzian FWHM */
    double irc_shift_rad;     /* Delta_M */
    double prins_g;           /* Darwin-Prins absorption parameter */
    double absorption_length_mm, absorption_ref_keV, absorption_power;
    double refl_K_per_mm2;    /* |r_e F_H / V| in mm^-2; < 0: derive from the Darwin width */
    double refl_darwin_fwhm_rad, refl_ref_keV;
    int64_t max_collisions;   /* per-ray cap on tentative collisions (STUCK) */
    double det_centre[3], det_u[3], det_v[3];
    int32_t det_nx, det_ny;
    double pixel_mm;
    /* candidate sampler of the walk: ORC_SAMPLER_PLAIN draws every tentative
     * collision at the constant majorant; ORC_SAMPLER_THINNED skips, per
     * straight segment, the candidates that provably cannot reflect (same
     * distribution of paths, fewer candidates).  thin_vstar: the acceptance
     * level below which every candidate is still tested (0: 2^-6). */
    int32_t sampler;
    int32_t pad3;
    double thin_vstar;
    /* higher-order reflections (Sec. 2.2.3: the cross-section is a sum over the
     * reflections H).  n_orders = 0: the single reflection on d_spacing_A.
     * Otherwise order h reflects on planes of spacing d_spacing_A / order_m[h],
     * with K_h = order_K_rel[h] K and a rocking curve order_w_rel[h] times as
     * wide as the one described above (same shape, same unit area). */
    int32_t n_orders, pad4;
    int32_t order_m[ORC_MAX_ORDERS];
    double order_K_rel[ORC_MAX_ORDERS], order_w_rel[ORC_MAX_ORDERS];
    /* energy-dependent rocking curve (Sec. 2.1 lets its width and peak shift be
     * functions of energy): width scale and an added shift at knots
     * irc_e_keV, linear between them, constant beyond; n_irc_e = 0: none */
    int32_t n_irc_e, pad5;
    double irc_e_keV[ORC_MAX_IRC_E], irc_e_wscale[ORC_MAX_IRC_E], irc_e_shift_rad[ORC_MAX_IRC_E];
} orc_spec;

enum { ORC_SAMPLER_PLAIN = 0, ORC_SAMPLER_THINNED = 1 };

typedef struct { int32_t kind; int32_t pad; double e0_keV, width_keV, lo_keV, hi_keV, weight; } orc_component;

typedef struct {
    int32_t n_comp; int32_t pad;
    orc_component comp[ORC_MAX_COMP];
    double origin[3], axis[3];
    double cone_half_angle_rad;
    double spot_fwhm_mm[2];
    double polarization[3];   /* linear polarisation p0 (projected perpendicular to
                                 each ray); zero vector: unpolarised */
    /* tabulated spectrum used by ORC_SRC_TABLE components: density values at
     * ascending knots; the CDF is the trapezoid-rule integral at the knots,
     * linear between them (a constant density within each interval) */
    const double *table_keV, *table_pdf;
    int32_t n_table, pad2;
} orc_source;

/* user-supplied rays (Sec. 2.1: origins, energies, directions and optional
 * polarisations given as arrays); px/py/pz may be NULL (unpolarised) */
typedef struct {
    const double *ox, *oy, *oz, *kx, *ky, *kz, *E, *px, *py, *pz;
} orc_rays;

typedef struct {
    uint64_t emitted, miss, absorbed, exit_front, exit_back, exit_side, capped, stuck,
             no_bragg, det_hits, refl_hist[16], collisions;
} orc_tally;

/* one record per traced ray (tests only) */
typedef struct {
    uint64_t ray_id;
    int32_t outcome, nrefl;
    int64_t ncoll;
    double energy_keV;
    double pos[3];            /* exit point, absorption point, or entry-less origin */
    double dir[3];            /* final direction */
    double u_mm, v_mm;        /* detector-plane coordinates (NaN if no plane hit) */
    int32_t ix, iy;           /* pixel (-1 if outside) */
    int32_t det_hit, no_bragg;
    double pol[3];            /* final polarisation (zero if unpolarised) */
} orc_record;

typedef struct {
    double body[ORC_MDF_M];       /* q = 1 - cos(theta) at u = i / M            */
    double tail[ORC_MDF_T + 1];   /* q at u = 1 - 2^-tau_j, tau_j = 12 + 21 j/T */
    double qmax;
} orc_mdf_table;

typedef struct {
    double E_keV, lambda_A, sin_aB, alpha_B, mu0, Q, mubar, p_abs;   /* sin_aB, alpha_B, Q: the first order */
    int32_t no_bragg, pad;                 /* no order has a Bragg solution */
    int32_t n_orders, pad2;
    double shift_rad;                      /* Delta_M(E) */
    /* per order: sin(alpha_B), alpha_B (NaN without a Bragg solution), Q, the
     * rocking-curve width scale, and Q R_max (its share of the majorant) */
    double ord_sin[ORC_MAX_ORDERS], ord_alpha[ORC_MAX_ORDERS], ord_Q[ORC_MAX_ORDERS];
    double ord_w[ORC_MAX_ORDERS], ord_qr[ORC_MAX_ORDERS];
} orc_ray_consts;

/* Philox4x32-10 (Salmon et al., SC'11) */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* pseudo-Voigt total width and eta (Sec. 2.2.1) */
void orc_pv_width(double fg, double fl, double *fwhm, double *eta);

/* IRC, unit area, argument = Delta - Delta_M (rad); ORC_IRC_NONE has no
 * finite value and returns 0 */
double orc_irc(const orc_spec *s, double x);
double orc_irc_max(const orc_spec *s);
double orc_darwin_prins_area(double g);       /* integral of R(y) dy */

/* MDF: un-normalised W as a function of q = 1 - cos(theta) */
double orc_mdf_W(const orc_spec *s, double q);
double orc_mdf_qmax(const orc_spec *s);
double orc_mdf_norm(const orc_spec *s);        /* integral of W dq over [0, qmax] */
double orc_mdf_cdf(const orc_spec *s, double q);      /* F(q) */
double orc_mdf_ccdf(const orc_spec *s, double q);     /* 1 - F(q), computed directly */
double orc_mdf_quantile_exact(const orc_spec *s, double u, int tail_complement, double comp);
int    orc_mdf_build_table(const orc_spec *s, orc_mdf_table *t);
double orc_mdf_table_lookup(const orc_mdf_table *t, uint32_t w);

/* per-ray constants (Eq. BraggLaw, Q of Sec. 2.2.3, majorant) */
int orc_ray_constants(const orc_spec *s, double E_keV, orc_ray_consts *c);

/* full path: source -> entry -> walk -> detector -> image (int64, += ) */
int orc_trace(const orc_spec *s, const orc_source *src, uint64_t n_rays, uint64_t seed,
              uint64_t ray_offset, int n_threads, int64_t *image, orc_tally *tally,
              orc_record *records);

/* detector quantum efficiency, linear in energy between the knots and
 * constant beyond them (Sec. 3: energies multiplied by their QE before the
 * keV image is binned); n = 0 means QE = 1 */
#define ORC_MAX_QE 32
typedef struct { int32_t n, pad; double keV[ORC_MAX_QE], qe[ORC_MAX_QE]; } orc_qe;
double orc_qe_eval(const orc_qe *q, double E_keV);

/* as orc_trace, and adds round(E * QE(E) * 1e6) (units of 1e-6 keV) of each
 * detected photon to energy_image (Sec. 2.3: the summed-keV image) */
int orc_trace_energy(const orc_spec *s, const orc_source *src, uint64_t n_rays, uint64_t seed,
                     uint64_t ray_offset, int n_threads, int64_t *image, int64_t *energy_image,
                     const orc_qe *qe, orc_tally *tally, orc_record *records);

/* as orc_trace_energy for user-supplied rays: ray i (id ray_offset + i) starts
 * at its own origin, direction, energy and polarisation; the walk draws its
 * Philox words from call 2 on, as for sampled rays */
int orc_trace_rays(const orc_spec *s, const orc_rays *rays, uint64_t n_rays, uint64_t seed,
                   uint64_t ray_offset, int n_threads, int64_t *image, int64_t *energy_image,
                   const orc_qe *qe, orc_tally *tally, orc_record *records);

/* the walk of one ray from a given entry state, fed with explicit 32-bit words
 * (4 per tentative collision) instead of Philox; for hand-traced tests */
int orc_walk_injected(const orc_spec *s, double E_keV, const double pos[3], const double dir[3],
                      const double *pol, const uint32_t *words, int64_t n_words, orc_record *rec);
/* n such walks sharing one mosaic table: ray i takes E[i], pos[3i..], dir[3i..],
 * pol[3i..] (pol may be NULL: all unpolarised) and words[i * words_per_ray ..] */
int orc_walk_injected_n(const orc_spec *s, int64_t n, const double *E_keV, const double *pos, const double *dir,
                        const double *pol, const uint32_t *words, int64_t words_per_ray, orc_record *rec);

/* accepted crystallites at a fixed ray direction and surface normal, first
 * reflection order: returns Delta (= alpha~ - alpha_B - Delta_M) and psi of n
 * accepted draws */
int64_t orc_sample_crystallites(const orc_spec *s, double E_keV, double alpha_rad, int64_t n,
                                uint64_t seed, double *delta_out, double *psi_out);

/* reflection rate r(alpha) (per mm of path) by 2-D quadrature of Eq. ReflXsection,
 * summed over the reflection orders */
double orc_reflection_rate(const orc_spec *s, double E_keV, double alpha_rad);

/* The thinned sampler's bounds of straight segments (test support): segment i
 * is a ray of energy E[i] at x[3i..] (inside or on the crystal) along
 * k[3i..], reflection order h; out[i] receives its bounds.  The
 * candidates the thinned walk never draws are those with v >= v* and either a
 * table word below w0 (tilt q below qmin), q above 2 - qmin, or an azimuth
 * outside the arcs where |k.n| lies in (S1, S2); without a rocking curve, the
 * facing cone's candidates outside |psi| < psis and the bounds wn, wf of
 * W / W(0) on the two cones.  Plain sampler or a segment near the Bragg angle:
 * ra = 1 (every candidate drawn). */
typedef struct {
    double s_exit;                /* distance to the first boundary crossing */
    int32_t face, thinned;        /* exit face; 1 if the thinned bounds apply to this order */
    double kN0, kN1;              /* k.N at the segment's start and exit */
    double xstar, vstar;          /* the spectrometer's X* (this order's width) and v* */
    double irc_max, W0, none_qv;  /* max R, W(0), the tilt beyond which W / W(0) <= v* */
    double alpha0;                /* aB + Delta_M of the order */
    double ra, qmin, pbar, S1, S2;
    uint64_t w0, wspan;
    double lam, mu, pa;           /* the order's candidate rate; the segment's majorant, mu0 / mu */
    double wn, wf, psis, pin, pio;
    uint64_t w1, w2;              /* one order: band B of process (b), table words [w1, w2) */
    double pbarB, sA;             /* band B's arc-measure bound; band A's share of process (b) */
} orc_seg_info;
int orc_segment_bounds(const orc_spec *s, int64_t n, const double *E_keV, const double *x, const double *k,
                       int h, orc_seg_info *out);

const char *orc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
