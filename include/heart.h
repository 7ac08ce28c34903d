/*
 * heart.h -- C ABI of the GB300 mosaic-crystal ray tracer.
 *
 * The library traces X-ray photons through a mosaic-crystal spectrometer as
 * described in Gawne et al., "HEART: A New X-Ray Tracing Code for Mosaic
 * Crystal Spectrometers" (arXiv 2503.16955): rays are sampled from a source
 * (Sec. 2.1), intersected with a flat or cylindrical (von Hamos) crystal
 * (Sec. 2.2), walked through the crystal depth with absorption and
 * mosaic-crystallite reflections (Sec. 2.2.3-2.2.4, Appendix A), and the rays
 * leaving the crystal are binned into integer detector pixels (Sec. 2.3).
 * Every step runs in CUDA kernels on the current device.
 *
 * Conventions
 *   Units: mm, keV, rad.  Vectors are 3 doubles in one global frame.
 *   Ownership: descriptors are host memory read during the call and not kept.
 *     Spectrometer tables live in device memory owned by the handle until
 *     heart_spectrometer_destroy.  Images passed to heart_trace are
 *     caller-owned device memory; the library adds counts (+=) and never
 *     clears them.  Server job images are owned by the server until
 *     heart_release.
 *   Errors: every call returns a heart_status; nothing throws across the ABI.
 *     heart_last_error() returns a thread-local message for the last failure
 *     in the calling thread.  Invalid descriptors, null or misaligned
 *     pointers return HEART_EINVAL before any launch.
 *   Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls on one spectrometer handle must not overlap in time
 *     (they share its tally scratch buffer): use one stream per handle or
 *     synchronise between calls.
 *   Determinism: each ray owns a Philox4x32-10 stream keyed by the seed and
 *     addressed by its ray id (ray_offset + i), so images and tallies do not
 *     depend on launch shape, chunking or concurrent jobs.
 */
#ifndef HEART_H
#define HEART_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HEART_OK = 0,
    HEART_EINVAL = 1,     /* bad argument or descriptor                      */
    HEART_ENOMEM = 2,     /* device or host allocation failed / over the cap */
    HEART_ECUDA = 3,      /* a CUDA runtime call failed                      */
    HEART_EBUSY = 4,      /* heart_poll: job not finished yet                */
    HEART_ETIMEOUT = 5,   /* heart_poll: timeout elapsed                     */
    HEART_ELIMIT = 6,     /* at least one ray hit the per-ray collision cap  */
    HEART_ENOTFOUND = 7   /* unknown job id                                  */
} heart_status;

typedef enum { HEART_FLAT = 0, HEART_CYL_VON_HAMOS = 1 } heart_geometry;

/* mosaic distribution functions W(theta) (Sec. 2.2.2) */
typedef enum {
    HEART_MDF_GAUSSIAN = 0,          /* Eq. (Gaussian) in theta               */
    HEART_MDF_LORENTZIAN = 1,        /* Eq. (Lorentz) in theta                */
    HEART_MDF_PSEUDO_VOIGT = 2,      /* eta L + (1 - eta) G, shared FWHM      */
    HEART_MDF_VMF = 3,               /* Eq. (MF), von Mises-Fisher            */
    HEART_MDF_WRAPPED_LORENTZIAN = 4,/* Eq. (WL)                              */
    HEART_MDF_SPHERICAL_WRAPPED_LORENTZIAN = 5, /* Eq. (SWL)                  */
    HEART_MDF_UNIFORM = 6            /* constant for theta <= Gamma / 2       */
} heart_mdf;

/* intrinsic rocking curves, unit area (Sec. 2.2.1) */
typedef enum {
    HEART_IRC_DARWIN = 0,            /* Darwin curve, FWHM = (3/sqrt 2) delta */
    HEART_IRC_DARWIN_PRINS = 1,      /* Darwin-Prins with absorption g        */
    HEART_IRC_PSEUDO_VOIGT = 2,      /* pseudo-Voigt from Gaussian/Lorentz FWHM */
    HEART_IRC_GAUSSIAN = 3,
    HEART_IRC_LORENTZIAN = 4,
    HEART_IRC_BOX = 5,
    /* no rocking curve (Sec. 2.2.1, "none"): R(Delta) = delta(Delta), so only
     * crystallites at exactly aB + Delta_M reflect (irc_fwhm_rad is ignored).
     * Candidates are drawn on the two Bragg cones k.n = -/+ sin(aB + Delta_M)
     * about the ray, at the rate Q cos(aB + Delta_M) 4 pi f(0) (f: the MDF per
     * unit solid angle), and kept with probability f(n) G / f(0); the sampler
     * field does not apply.  The cost per ray grows as 1 / Gamma^2 for narrow
     * mosaics. */
    HEART_IRC_NONE = 6
} heart_irc;

typedef enum { HEART_FP64 = 0, HEART_FP32 = 1 } heart_precision;

/* Candidate sampler of the depth walk.  THINNED (the default) never draws,
 * per straight segment, the tentative collisions that provably cannot reflect
 * (crystallite tilts and azimuths whose |Delta| exceeds the rocking curve's
 * half-width X* at relative level v*): the same distribution of paths as
 * PLAIN, the constant-majorant walk of Sec. 2.2.3-2.2.4, with several times
 * fewer candidates off the Bragg angle.  With one reflection order the
 * candidates that may reflect are drawn in two tilt bands, each at its own bound
 * of the azimuth measure that reaches the Bragg window (fewer again by half). */
typedef enum { HEART_SAMPLER_THINNED = 0, HEART_SAMPLER_PLAIN = 1 } heart_sampler;
typedef enum { HEART_COUNT_I32 = 0, HEART_COUNT_I64 = 1 } heart_count_type;

/* spectral component kinds (Sec. 2.1: an intensity profile used as a PDF) */
typedef enum {
    HEART_SRC_MONO = 0,      /* delta at e0                               */
    HEART_SRC_GAUSS = 1,     /* Gaussian, sigma = width                   */
    HEART_SRC_LORENTZ = 2,   /* Lorentzian, FWHM = width, truncated E > 0 */
    HEART_SRC_INV_E = 3,     /* 1/E on [lo, hi]                           */
    HEART_SRC_UNIFORM = 4,   /* uniform on [lo, hi]                       */
    HEART_SRC_TABLE = 5      /* the source's tabulated spectrum (below)    */
} heart_source_kind;

/* ray outcomes (Sec. 2.2.4) */
typedef enum {
    HEART_MISS = 0, HEART_ABSORBED = 1, HEART_EXIT_FRONT = 2, HEART_EXIT_BACK = 3,
    HEART_EXIT_SIDE = 4, HEART_CAPPED = 5, HEART_STUCK = 6
} heart_outcome;

typedef struct heart_spectrometer heart_spectrometer;
typedef struct heart_server heart_server;

/*
 * Crystal and detector (Sec. 2.2 crystal classes, Sec. 2.3 detector).
 * Flat: the crystal occupies the slab -thickness <= (x - centre).N <= 0,
 *   |(x - centre).e_d| <= size_disp/2, |(x - centre).(N x e_d)| <= size_nondisp/2,
 *   with N = normal and e_d = axis projected perpendicular to N.
 * Cylindrical (von Hamos): the shell R <= r <= R + thickness around the line
 *   through `centre` along `axis`; axial coordinate within
 *   centre_axial +- size_disp/2; azimuth within +- size_nondisp/(2R) of the
 *   direction `normal` (projected perpendicular to the axis).  The inner face
 *   r = R reflects; the local normal points toward the axis.
 * Detector: plane through det_centre spanned by det_u, det_v (orthonormalised);
 *   pixel (ix, iy) = floor(u/pixel + nx/2), floor(v/pixel + ny/2); either face.
 */
typedef struct {
    double d_spacing_A;             /* lattice spacing d_H, Eq. (BraggLaw)     */
    double thickness_mm;
    int32_t geometry;               /* heart_geometry */
    int32_t mdf;                    /* heart_mdf */
    double radius_mm;               /* cylinder radius (inner face)            */
    double centre_mm[3];
    double normal[3];
    double axis[3];
    double centre_axial_mm;         /* cylinder only */
    double size_disp_mm, size_nondisp_mm;
    double mdf_fwhm_rad;            /* Gamma */
    double mdf_eta;                 /* pseudo-Voigt MDF Lorentzian fraction */
    int32_t irc;                    /* heart_irc */
    int32_t max_reflections;        /* the (n+1)-th reflection ends the ray as CAPPED */
    double irc_fwhm_rad;            /* Darwin/DP: Darwin FWHM; G/L/box: FWHM; pV: Gaussian FWHM; none: unused */
    double irc_lorentz_fwhm_rad;    /* pV: Lorentzian FWHM */
    double irc_shift_rad;           /* Delta_M, peak position of the IRC */
    double prins_g;                 /* Darwin-Prins absorption parameter */
    double absorption_length_mm;    /* 1/mu0 at absorption_ref_keV */
    double absorption_ref_keV;
    double absorption_power;        /* l_abs(E) = l_ref (E / E_ref)^power */
    double refl_K_per_mm2;          /* K = |r_e F_H / V|; < 0: derive from refl_darwin_fwhm_rad */
    double refl_darwin_fwhm_rad;    /* Darwin FWHM at refl_ref_keV (used when K < 0) */
    double refl_ref_keV;
    int64_t max_collisions;         /* per-ray cap on tentative collisions (STUCK) */
    double det_centre_mm[3], det_u[3], det_v[3];
    int32_t det_nx, det_ny;
    double pixel_mm;
    int32_t count_type;             /* heart_count_type of images traced with this handle */
    int32_t sampler;                /* heart_sampler */
    double thin_vstar;              /* THINNED: relative IRC level v* in (0, 1); 0: 2^-6 */
    /* Higher-order reflections (Sec. 2.2.3: the cross-section is a sum over the
     * reflections H, e.g. graphite (002), (004), (006)).  n_orders = 0: the
     * single reflection on d_spacing_A.  Otherwise order h reflects on planes
     * d_spacing_A / order_m[h] with K_h = order_K_rel[h] K and a rocking curve
     * order_w_rel[h] times as wide (same shape and unit area).  A scatter
     * candidate picks its order by the order's share of the candidate rate.
     * Both precisions take up to HEART_MAX_ORDERS.  FP32 traces of sampled
     * sources with several orders run on the two-pass trace; user-supplied
     * rays with several orders, and batched jobs below 2^18 rays, on the
     * persistent kernel. */
    int32_t n_orders;
    int32_t reserved2;
    int32_t order_m[4];
    double order_K_rel[4], order_w_rel[4];
    /* Energy-dependent rocking curve (Sec. 2.1: its width and peak shift as
     * functions of energy): at the ascending knots irc_e_keV the width scale
     * irc_e_wscale (> 0) and a shift irc_e_shift_rad added to irc_shift_rad,
     * linear between knots and constant beyond them; n_irc_e = 0: none. */
    int32_t n_irc_e;
    int32_t reserved3;
    double irc_e_keV[16], irc_e_wscale[16], irc_e_shift_rad[16];
} heart_spectrometer_desc;

#define HEART_MAX_ORDERS 4
#define HEART_MAX_IRC_E 16

typedef struct {
    int32_t kind;                   /* heart_source_kind */
    int32_t reserved;
    double e0_keV, width_keV, lo_keV, hi_keV;
    double weight;                  /* relative photon share of this component */
} heart_spectral_component;

/* Point or Gaussian-spot source emitting uniformly in solid angle inside a cone. */
typedef struct {
    const heart_spectral_component *components;   /* host array, 1..16 entries */
    int32_t n_components;
    int32_t reserved;
    double origin_mm[3];
    double axis[3];                 /* cone axis */
    double cone_half_angle_rad;
    double spot_fwhm_mm[2];         /* 2-D Gaussian spot perpendicular to the axis */
    double polarization[3];         /* linear polarisation p0, projected perpendicular to each
                                       ray (Sec. 2.1); zero vector: unpolarised */
    /* Tabulated spectrum (Sec. 2.1: a measured or modelled spectrum), drawn by
     * components of kind HEART_SRC_TABLE: density values table_pdf[i] >= 0 at
     * strictly ascending energies table_keV[i] > 0, 2 <= n_table <= 8192 (host
     * arrays, copied during the call).  The CDF is the trapezoid rule at the
     * knots and linear between them (constant density inside an interval).
     * NULL / 0 when no component uses it. */
    const double *table_keV;
    const double *table_pdf;
    int32_t n_table;
    int32_t reserved2;
} heart_source_desc;

#define HEART_MAX_TABLE 8192

/* User-supplied rays (Sec. 2.1: origins, energies, directions and optional
 * polarisations instead of a sampled source).  Device arrays of n doubles
 * each (structure of arrays, read coalesced); directions need not be
 * normalised; pol_* may all be NULL (unpolarised), otherwise each is
 * projected perpendicular to its ray.  Ray i has id ray_offset + i. */
typedef struct {
    const double *origin_x, *origin_y, *origin_z;
    const double *dir_x, *dir_y, *dir_z;
    const double *energy_keV;
    const double *pol_x, *pol_y, *pol_z;
} heart_ray_arrays;

/* Detector quantum efficiency (Sec. 3): QE(E) linear between the knots,
 * constant beyond the first and last; keV strictly increasing, 1..32 knots,
 * qe in [0, 1]. */
typedef struct {
    const double *keV;              /* host array, n entries */
    const double *qe;               /* host array, n entries */
    int32_t n;
    int32_t reserved;
} heart_qe_table;

typedef struct {
    uint64_t emitted, miss, absorbed, exit_front, exit_back, exit_side, capped, stuck;
    uint64_t no_bragg, det_hits;
    uint64_t refl_hist[16];         /* rays that entered, by reflections (15 = 15 or more) */
    uint64_t collisions;            /* tentative collisions (null-collision walk steps inside) */
} heart_tally;

/* per-ray record (tests and debugging) */
typedef struct {
    uint64_t ray_id;
    int32_t outcome, nrefl;
    int64_t ncoll;
    double energy_keV;
    double pos[3];                  /* exit or absorption point; source origin for MISS */
    double dir[3];
    double u_mm, v_mm;              /* detector-plane coordinates, NaN if the plane is not hit */
    int32_t ix, iy;                 /* pixel, -1 outside */
    int32_t det_hit, no_bragg;
    double pol[3];                  /* final polarisation, zero if unpolarised */
} heart_ray_record;

/* Create a spectrometer: validates the descriptor, builds the mosaic
 * inverse-CDF table and IRC constants on the current device.  Returns
 * HEART_EINVAL for an invalid descriptor, HEART_ENOMEM / HEART_ECUDA on
 * device failures. */
heart_status heart_spectrometer_create(const heart_spectrometer_desc *desc, heart_spectrometer **out);
heart_status heart_spectrometer_destroy(heart_spectrometer *spec);

/* Trace rays ray_offset .. ray_offset + n_rays - 1 (Sec. 2.2.4: n_rays counts
 * emitted rays, misses included) and add their detector hits to d_image
 * (device, det_ny x det_nx row-major, int32 or int64 per the descriptor,
 * aligned to its element size).  precision selects the plain FP64 kernel or
 * the FP32 kernels.  If `out` is non-NULL the call synchronises `stream` and
 * fills the tallies; returns HEART_ELIMIT (after filling) if a ray hit the
 * collision cap.  FP32 image traces (all but user rays with several reflection
 * orders) run in two passes through a hit queue that the library keeps per
 * device for the process (two buffers, up to 15 GB, allocated on first use,
 * shared by all spectrometers; such traces run one after another on the GPU
 * whatever their streams, each on `stream` and a side stream of the library's
 * that `stream` waits for before the call's work ends). */
heart_status heart_trace(heart_spectrometer *spec, const heart_source_desc *src, uint64_t n_rays,
                         uint64_t seed, uint64_t ray_offset, void *d_image,
                         heart_precision precision, void *stream, heart_tally *out);

/* As heart_trace, and also adds each detected photon's energy times the
 * detector quantum efficiency QE(E) to d_energy_image (device, uint64,
 * det_ny x det_nx, 8-byte aligned, += ) in units of 1e-6 keV, rounded to the
 * nearest unit per photon so sums do not depend on order (the summed-keV image
 * of Sec. 2.3, QE of Sec. 3).  qe may be NULL (QE = 1).  d_image may be NULL
 * when only the energy image is wanted; the counts then go to a scratch image
 * of the handle.  Energy image / count image is the calibration map of a
 * uniform spectrum (Sec. 3). */
heart_status heart_trace_energy(heart_spectrometer *spec, const heart_source_desc *src, uint64_t n_rays,
                                uint64_t seed, uint64_t ray_offset, void *d_image, uint64_t *d_energy_image,
                                const heart_qe_table *qe, heart_precision precision, void *stream,
                                heart_tally *out);

/* Calibration map of the detector (Sec. 3: the energy dispersion of a
 * spectrometer, traced with a flat spectrum): the geometry of `src` (origin,
 * cone, spot, polarisation; its spectral components are ignored) with one
 * uniform component on [min_keV, max_keV], traced as heart_trace_energy with
 * QE = 1 into d_counts (the handle's count type) and d_energy_image (uint64,
 * 1e-6 keV units), both device, det_ny x det_nx, added to (+=); then
 * d_mean_keV (device, double, det_ny x det_nx, overwritten) receives each
 * pixel's mean energy, energy / counts, NaN where no photon landed.  Pass
 * zeroed images for a map of this trace alone.  If `out` is non-NULL the call
 * synchronises and fills the tallies. */
heart_status heart_calibration_map(heart_spectrometer *spec, const heart_source_desc *src, double min_keV,
                                   double max_keV, uint64_t n_rays, uint64_t seed, heart_precision precision,
                                   void *d_counts, uint64_t *d_energy_image, double *d_mean_keV, void *stream,
                                   heart_tally *out);

/* Trace user-supplied rays (heart_ray_arrays, device memory) instead of a
 * sampled source; the walk, detector and tallies are those of heart_trace.
 * Polarised rays use G = 1 - (p . k_s)^2 (Eq. G_pol) and the polarisation
 * update of Sec. 2.2.4.  d_records (device, n_rays heart_ray_record, may be
 * NULL) receives one record per ray; the call then synchronises. */
heart_status heart_trace_rays(heart_spectrometer *spec, const heart_ray_arrays *rays, uint64_t n_rays,
                              uint64_t seed, uint64_t ray_offset, void *d_image, heart_precision precision,
                              void *d_records, void *stream, heart_tally *out);

/* As heart_trace, with host memory: h_image (host, += ) is copied to the
 * device, traced and copied back inside the call.  Synchronous. */
heart_status heart_trace_host(heart_spectrometer *spec, const heart_source_desc *src,
                              uint64_t n_rays, uint64_t seed, uint64_t ray_offset, void *h_image,
                              heart_precision precision, heart_tally *out);

/* As heart_trace, and also writes one heart_ray_record per ray to d_records
 * (device, n_rays entries).  d_image may be NULL.  Synchronous. */
heart_status heart_trace_records(heart_spectrometer *spec, const heart_source_desc *src,
                                 uint64_t n_rays, uint64_t seed, uint64_t ray_offset,
                                 void *d_image, heart_precision precision, void *d_records,
                                 void *stream, heart_tally *out);

/* Many spectrometers of uneven ray counts, FP32, on `stream`.  Jobs of fewer
 * than 2^18 rays share one persistent
 * launch (work items = (job, ray range) claimed by blocks); larger jobs run as
 * single-job two-pass traces, as heart_trace runs them, so a large job's image
 * and tallies equal its single trace.  specs[i], srcs[i], n_rays[i], seeds[i],
 * d_images[i] describe job i; out (may be NULL) receives n_jobs tallies after a
 * stream synchronisation.  Allocates a small per-call work area, and the
 * device's hit queue for the two-pass trace if it is not large enough yet. */
heart_status heart_trace_batch(heart_spectrometer *const *specs, const heart_source_desc *const *srcs,
                               const uint64_t *n_rays, const uint64_t *seeds, void *const *d_images,
                               int32_t n_jobs, void *stream, heart_tally *out);

/* Launch shape of the FP32 kernels chosen by heart_autotune. */
typedef struct {
    int32_t blocks_per_sm;          /* persistent kernel: resident 128-thread blocks per SM, 6 (80
                                       registers) or 5 (96; the default before any autotune) */
    int32_t refill_lanes;           /* a warp takes queued or spawned rays when this many lanes are idle */
    uint32_t max_chunk_rays;        /* largest work item (rays) a block of the persistent kernel claims */
    int32_t reserved;
    double rays_per_s;              /* this trace's rate on the probe with the chosen refill threshold */
} heart_tune;

/* Time FP32 traces of probe_rays rays of this spectrometer and source: first
 * the refill threshold (1, 4, 8 or 16 idle lanes) on the path this trace takes
 * (the two-pass trace for image traces it covers), then the persistent
 * kernel's blocks per SM (6 or 5), which batched jobs below 2^18 rays and
 * served slices use, on that kernel.  The fastest choices hold for all later
 * FP32 launches of the process.  Call it before tracing, not concurrently with
 * traces.  Uses the handle's scratch image; `out` (may be NULL) receives the
 * choice. */
heart_status heart_autotune(heart_spectrometer *spec, const heart_source_desc *src, uint64_t probe_rays,
                            void *stream, heart_tune *out);

/* Maximum number of jobs of heart_trace_batch_static. */
#define HEART_STATIC_MAX_JOBS 64

/* heart_trace_batch for callers that cannot allocate device memory during the
 * call (this entry point has no counterpart in the paper; it exists for
 * deployment).  Examples: an application that gives all free device memory
 * to its own pool at start-up, or a control loop that must not risk an
 * allocation failure or the synchronisation an allocation can cause.
 * heart_trace_batch allocates a small per-call work area (job table, work
 * counter, tallies); this variant uses a fixed work area in a device array
 * that the library declares at file scope, sized for HEART_STATIC_MAX_JOBS
 * jobs, and allocates nothing on the device.  The caller still passes the
 * spectrometers (created beforehand), sources and device images, as for
 * heart_trace_batch, and gets the same images and tallies: every job runs on
 * the persistent kernel here (the two-pass trace needs the hit queue), which
 * traces each ray as the two-pass trace does.
 *   - n_jobs > HEART_STATIC_MAX_JOBS returns HEART_EINVAL with a message.
 *   - Sources with a tabulated-spectrum component (HEART_SRC_TABLE) return
 *     HEART_EINVAL: their table needs a device copy this call cannot make.
 *   - Every GPU that loads the library holds the array until the process exits.
 *   - All calls share the array; each call rewrites it (tallies and the work
 *     counter start at zero), so calls that overlap on the GPU race: serialise
 *     them on one stream.  Host staging is serialised by a lock.
 *   - The work area is uploaded from pageable host memory, so the call may
 *     wait for earlier work on `stream` before it returns.
 *   - The first call on each device looks up the array's device address (with
 *     that device current).
 * If `out` is non-NULL the call synchronises `stream` and fills n_jobs tallies. */
heart_status heart_trace_batch_static(heart_spectrometer *const *specs, const heart_source_desc *const *srcs,
                                      const uint64_t *n_rays, const uint64_t *seeds, void *const *d_images,
                                      int32_t n_jobs, void *stream, heart_tally *out);

/* Request loop (continuous batching): jobs are admitted in arrival order while
 * their images fit under mem_cap_bytes and stay resident until released.  A
 * worker thread keeps two rounds of launches in flight; each round traces, in
 * arrival order, every admitted job with at most 2^20 rays left whole, and
 * gives a budget of 2^26 rays to the larger ones oldest first in slices of at
 * least 2^22 rays.  Slices of 2^18 rays or more run as two-pass traces, the
 * others together in one persistent batched launch; every FP32 kernel traces a
 * ray alike, so a job's image and tallies equal its heart_trace's. */
heart_status heart_server_create(size_t mem_cap_bytes, heart_server **out);
heart_status heart_server_destroy(heart_server *server);
heart_status heart_submit(heart_server *server, heart_spectrometer *spec, const heart_source_desc *src,
                          uint64_t n_rays, uint64_t seed, heart_precision precision, uint64_t *job_id);
/* HEART_OK when done (tallies and a device image pointer valid until
 * heart_release), HEART_ETIMEOUT if not done within timeout_ms (0 = do not
 * wait, returns HEART_EBUSY), HEART_ENOTFOUND for an unknown id. */
heart_status heart_poll(heart_server *server, uint64_t job_id, int32_t timeout_ms, heart_tally *out,
                        const void **d_image_out);
heart_status heart_release(heart_server *server, uint64_t job_id);
/* Copy a finished job's image (det_ny x det_nx, the handle's count type) into
 * dst: host memory if dst_is_host != 0, else device memory.  Synchronous. */
heart_status heart_fetch_image(heart_server *server, uint64_t job_id, void *dst, int32_t dst_is_host);
/* Seconds from heart_submit to completion, measured by the server (finished jobs). */
heart_status heart_job_latency(heart_server *server, uint64_t job_id, double *seconds);

/* Issue rates of the SM pipes the ray path runs on (measurement support; the
 * paper has no counterpart).  The ray kernels issue integer (Philox), FP32 and
 * SFU instructions and are bound by those pipes, not by memory, so their
 * roofline is the rate each pipe sustains.  heart_pipe_peaks runs one
 * microbenchmark kernel per instruction below (eight dependent chains per
 * thread, 32 resident warps per SM, inline PTX so the instruction is the one
 * named) and reports, per instruction, warp instructions per second for the
 * whole GPU (CUDA events) and per SM per clock (clock64 in every block), and
 * the mean SM clock the runs saw.  It takes about 0.1 s, allocates a few MB
 * of device memory for its own use and synchronises `stream`. */
enum {
    HEART_PIPE_FFMA = 0,       /* fma.rn.f32                       */
    HEART_PIPE_LOP3 = 1,       /* lop3.b32 (three-input logic)     */
    HEART_PIPE_IADD3 = 2,      /* add.u32                          */
    HEART_PIPE_IMAD = 3,       /* mad.lo.u32                       */
    HEART_PIPE_IMAD_HI = 4,    /* mul.hi.u32 (Philox's multiply)   */
    HEART_PIPE_IMAD_WIDE = 5,  /* mul.wide.u32                     */
    HEART_PIPE_MUFU_RSQ = 6,   /* rsqrt.approx.ftz.f32 (SFU)       */
    HEART_PIPE_MUFU_EX2 = 7,   /* ex2.approx.ftz.f32 (SFU)         */
    HEART_PIPE_MUFU_LG2 = 8,   /* lg2.approx.ftz.f32 (SFU)         */
    HEART_PIPE_DFMA = 9,       /* fma.rn.f64                       */
    HEART_PIPE_NOPS = 10
};
typedef struct {
    double warp_inst_per_s[HEART_PIPE_NOPS];      /* whole GPU, at the clocks of the run */
    double warp_inst_per_clk_sm[HEART_PIPE_NOPS]; /* per SM per SM clock                 */
    double sm_clock_hz;                           /* mean SM clock during the runs        */
    int32_t sms;
    int32_t n_ops;
} heart_pipe_rates;
heart_status heart_pipe_peaks(void *stream, heart_pipe_rates *out);

/* Test support (no counterpart in the paper): device functions of the FP32
 * kernels evaluated on n values of the device arrays d_x (and d_y, d_z),
 * results in d_out (device, n floats); asynchronous on `stream`.  which = 0:
 * the arccos of the azimuth arcs, acos(x / y) for y > 0 (spec may be NULL,
 * d_z unused); 1: the spectrometer's rocking curve divided by its maximum,
 * R(x) / R_max at x = Delta - Delta_M; 2: the upper bound of R / R_max over
 * |x'| >= x that the kernels' early rejection uses (1 and 2 need spec, read
 * d_x only); 3: the upper bound the walk places on the measure, in units of
 * pi, of the azimuth arc with cos(xi') in (x, y) / z (z > 0); 4: that measure
 * as the thinned sampler computes it (3 and 4: spec may be NULL).  Null
 * arrays the function reads, or which outside 0..4, give HEART_EINVAL. */
heart_status heart_check_functions(heart_spectrometer *spec, int32_t which, const float *d_x, const float *d_y,
                                   const float *d_z, float *d_out, uint64_t n, void *stream);

const char *heart_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
