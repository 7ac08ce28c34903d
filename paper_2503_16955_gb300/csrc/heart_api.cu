// heart_api.cu -- the C ABI entry points and the plain FP64 kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "heart.h"
#include "heart_fp64.cuh"
#include "heart_internal.h"
#include "heart_lib.h"

namespace heart {

thread_local std::string g_last_error;

heart_status fail(heart_status st, const char *msg) {
    g_last_error = msg;
    return st;
}

heart_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return HEART_ECUDA;
}

// ---------------------------------------------------------------------------
// plain FP64 kernel: one ray per thread, grid-stride, mosaic table in smem
// ---------------------------------------------------------------------------
template <typename CountT>
__device__ __forceinline__ void add_pixel(CountT *img, size_t idx);
template <>
__device__ __forceinline__ void add_pixel<int32_t>(int32_t *img, size_t idx) { atomicAdd((int *)img + idx, 1); }
template <>
__device__ __forceinline__ void add_pixel<int64_t>(int64_t *img, size_t idx) {
    atomicAdd((unsigned long long *)img + idx, 1ull);
}

__device__ __forceinline__ double qe64(const QeParams &Q, double E) {
    if (Q.n <= 0) return 1.0;
    if (E <= Q.keV[0]) return Q.qe[0];
    for (int i = 1; i < Q.n; ++i)
        if (E <= Q.keV[i]) {
            const double f = (E - Q.keV[i - 1]) / (Q.keV[i] - Q.keV[i - 1]);
            return Q.qe[i - 1] + f * (Q.qe[i] - Q.qe[i - 1]);
        }
    return Q.qe[Q.n - 1];
}

template <typename CountT>
__global__ void __launch_bounds__(256) k_trace_fp64(const SpecParams S, const SourceParams P, uint64_t n,
                                                    uint32_t k0, uint32_t k1, uint64_t offset, CountT *img,
                                                    unsigned long long *tally, heart_ray_record *rec,
                                                    const __grid_constant__ QeParams Q) {
    extern __shared__ double s_tab[];
    __shared__ unsigned long long s_t[kTallyN];
    for (int i = threadIdx.x; i < kMdfKnots; i += blockDim.x) s_tab[i] = S.mdf64[i];
    for (int i = threadIdx.x; i < kTallyN; i += blockDim.x) s_t[i] = 0ull;
    __syncthreads();
    unsigned long long my_emit = 0, my_coll = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        RayOut64 r;
        trace_ray64(S, P, k0, k1, offset + i, i, s_tab, r);
        ++my_emit;
        my_coll += (unsigned long long)r.ncoll;
        atomicAdd(&s_t[r.outcome == HEART_MISS ? T_MISS : T_ABSORBED + (r.outcome - HEART_ABSORBED)], 1ull);
        if (r.outcome != HEART_MISS) atomicAdd(&s_t[T_HIST0 + (r.nrefl < 15 ? r.nrefl : 15)], 1ull);
        if (r.no_bragg) atomicAdd(&s_t[T_NO_BRAGG], 1ull);
        if (r.det_hit) {
            const size_t idx = (size_t)r.iy * (size_t)S.nx + (size_t)r.ix;
            add_pixel<CountT>(img, idx);
            atomicAdd(&s_t[T_DET_HITS], 1ull);
            if (Q.eimg) atomicAdd(Q.eimg + idx, (unsigned long long)llrint(r.E * qe64(Q, r.E) * 1e6));
        }
        if (rec) {
            heart_ray_record &o = rec[i];
            o.ray_id = offset + i;
            o.outcome = r.outcome;
            o.nrefl = r.nrefl;
            o.ncoll = r.ncoll;
            o.energy_keV = r.E;
            for (int j = 0; j < 3; ++j) { o.pos[j] = r.pos[j]; o.dir[j] = r.dir[j]; }
            o.u_mm = r.u;
            o.v_mm = r.v;
            o.ix = r.ix;
            o.iy = r.iy;
            o.det_hit = r.det_hit;
            o.no_bragg = r.no_bragg;
            for (int j = 0; j < 3; ++j) o.pol[j] = r.pol[j];
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        my_emit += __shfl_down_sync(0xffffffffu, my_emit, off);
        my_coll += __shfl_down_sync(0xffffffffu, my_coll, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_t[T_EMITTED], my_emit);
        atomicAdd(&s_t[T_COLLISIONS], my_coll);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTallyN; i += blockDim.x)
        if (s_t[i]) atomicAdd(&tally[i], s_t[i]);
}

static int g_num_sms = 0;
int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

heart_status launch_fp64(const SpecParams &S, const SourceParams &P, uint64_t n, uint64_t seed, uint64_t offset,
                         void *img, unsigned long long *tally, heart_ray_record *rec, cudaStream_t st,
                         const QeParams *qe) {
    if (n == 0) return HEART_OK;
    QeParams Q;
    if (qe) Q = *qe;
    else std::memset(&Q, 0, sizeof Q);
    const int threads = 256;
    const size_t smem = (size_t)kMdfKnots * sizeof(double);
    uint64_t want = (n + threads - 1) / threads;
    uint64_t cap = (uint64_t)num_sms() * 6;
    const int blocks = (int)(want < cap ? want : cap);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    if (S.count_type == HEART_COUNT_I64) {
        static bool attr = false;
        if (!attr) { cudaFuncSetAttribute(k_trace_fp64<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); attr = true; }
        k_trace_fp64<int64_t><<<blocks, threads, smem, st>>>(S, P, n, k0, k1, offset, (int64_t *)img, tally, rec, Q);
    } else {
        static bool attr = false;
        if (!attr) { cudaFuncSetAttribute(k_trace_fp64<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); attr = true; }
        k_trace_fp64<int32_t><<<blocks, threads, smem, st>>>(S, P, n, k0, k1, offset, (int32_t *)img, tally, rec, Q);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "FP64 kernel launch");
    return HEART_OK;
}

}  // namespace heart

using namespace heart;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" const char *heart_last_error(void) { return g_last_error.c_str(); }

// X*: the smallest |x| with R(x') / R_max <= v* for all |x'| >= X* (the
// rocking curves are even and fall off monotonically outside their core):
// walk |x| down from 1 rad in steps of 1/2000 relative until R / R_max
// exceeds v*, bisect that step, widen the result by 1e-6 relative
static double rocking_half_width(const SpecParams &S) {
    auto rel = [&](double x) { return irc64(S, x) / S.irc_max; };
    double x = 1.0;
    if (rel(x) > S.vstar) return -1.0;
    for (;;) {
        const double y = x / 1.0005;
        if (y < 1e-12) return 1e-12;
        if (rel(y) > S.vstar) {
            double lo = y, hi = x;
            for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
                const double m = 0.5 * (lo + hi);
                if (rel(m) > S.vstar) lo = m; else hi = m;
            }
            return hi * (1.0 + 1e-6);
        }
        x = y;
    }
}

extern "C" heart_status heart_spectrometer_create(const heart_spectrometer_desc *desc, heart_spectrometer **out) {
    if (!out) return fail(HEART_EINVAL, "null output pointer");
    *out = nullptr;
    std::vector<double> tab(kMdfKnots);
    SpecParams p;
    char err[256] = {0};
    heart_status st = build_spec_params(desc, &p, tab.data(), err, (int)sizeof err);
    if (st != HEART_OK) return fail(st, err);
    if (p.sampler == HEART_SAMPLER_THINNED && p.irc != HEART_IRC_NONE) {
        p.xstar = rocking_half_width(p);
        if (!(p.xstar > 0)) return fail(HEART_EINVAL, "rocking curve does not fall below v* within 1 rad");
    }
    std::vector<float> tab32(kMdfKnots);
    for (int i = 0; i < kMdfKnots; ++i) tab32[i] = (float)tab[i];
    heart_spectrometer *h = new (std::nothrow) heart_spectrometer();
    if (!h) return fail(HEART_ENOMEM, "host allocation failed");
    cudaError_t e;
    if ((e = cudaGetDevice(&h->device)) != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
    // thinned sampler: first table word of the interval holding each grid point
    // q_j = 2^(j/8 - 48) (the body knots are ascending; at or past the last one: the tail)
    std::vector<uint32_t> qgrid(kQGrid);
    for (int j = 0; j < kQGrid; ++j) {
        const double q = std::exp2(j / 8.0 - 48.0);
        uint32_t w = (uint32_t)(kMdfM - 1) << 20;
        if (q < tab[kMdfM - 1]) {
            int lo = 0, hi = kMdfM - 1;
            if (!(tab[0] <= q)) { lo = 0; hi = 0; }
            while (hi - lo > 1) {
                const int m = (lo + hi) / 2;
                if (tab[m] <= q) lo = m; else hi = m;
            }
            w = (uint32_t)lo << 20;
        }
        qgrid[j] = w;
    }
    // band B of process (b): 1 / sin(theta) at the knot starting each grid word's interval
    std::vector<float> is1(kQGrid);
    for (int j = 0; j < kQGrid; ++j) {
        const double q = tab[qgrid[j] >> 20];
        const double st = std::sqrt(q * (2.0 - q));
        is1[j] = st > 0.0 ? std::nextafter((float)(1.0 / st), INFINITY) : 0.0f;
    }
    // [FP64 table][FP32 table, padded to 8 bytes][scratch words][tilt grid words][band B 1 / sin]
    size_t bytes = kMdfKnots * sizeof(double) + (kMdfKnots + (kMdfKnots & 1)) * sizeof(float) +
                   kScratchWords * sizeof(unsigned long long) + kQGrid * sizeof(uint32_t) + kQGrid * sizeof(float);
    if ((e = cudaMalloc(&h->d_block, bytes)) != cudaSuccess) { delete h; return cuda_fail(e, "cudaMalloc tables"); }
    h->d_tab64 = (double *)h->d_block;
    h->d_tab32 = (float *)(h->d_tab64 + kMdfKnots);
    h->d_scratch = (unsigned long long *)(h->d_tab32 + kMdfKnots + (kMdfKnots & 1));
    uint32_t *d_qgrid = (uint32_t *)(h->d_scratch + kScratchWords);
    float *d_is1 = (float *)(d_qgrid + kQGrid);
    if ((e = cudaMemcpy(h->d_tab64, tab.data(), kMdfKnots * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(h->d_tab32, tab32.data(), kMdfKnots * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d_qgrid, qgrid.data(), kQGrid * sizeof(uint32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(d_is1, is1.data(), kQGrid * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(h->d_block);
        delete h;
        return cuda_fail(e, "cudaMemcpy tables");
    }
    if ((e = cudaMallocHost(&h->h_scratch, kScratchWords * sizeof(unsigned long long))) != cudaSuccess) {
        cudaFree(h->d_block);
        delete h;
        return cuda_fail(e, "cudaMallocHost");
    }
    p.mdf64 = h->d_tab64;
    p.mdf32 = h->d_tab32;
    p.qgrid = d_qgrid;
    p.band_w2 = qgrid[kBandJ2];
    p.band_is1 = d_is1;
    h->p = p;
    h->desc = *desc;
    *out = h;
    return HEART_OK;
}

extern "C" heart_status heart_spectrometer_destroy(heart_spectrometer *h) {
    if (!h) return fail(HEART_EINVAL, "null spectrometer");
    cudaFree(h->d_block);
    cudaFreeHost(h->h_scratch);
    if (h->d_image_host_path) cudaFree(h->d_image_host_path);
    delete h;
    return HEART_OK;
}

static void fill_tally(const unsigned long long *t, heart_tally *out) {
    std::memcpy(out, t, sizeof(heart_tally));
}

// common body of heart_trace / heart_trace_records / heart_trace_energy / heart_trace_rays
static heart_status trace_impl(heart_spectrometer *h, const heart_source_desc *src, uint64_t n_rays, uint64_t seed,
                               uint64_t ray_offset, void *d_image, heart_precision prec, void *d_records,
                               void *stream, heart_tally *out, bool sync, const QeParams *qe = nullptr,
                               const SourceParams *prepared = nullptr) {
    if (!h) return fail(HEART_EINVAL, "null spectrometer");
    if (prec != HEART_FP64 && prec != HEART_FP32) return fail(HEART_EINVAL, "unknown precision");
    size_t elt = h->p.count_type == HEART_COUNT_I64 ? 8 : 4;
    if (!d_image && !d_records && !(qe && qe->eimg)) return fail(HEART_EINVAL, "null image");
    if (d_image && ((uintptr_t)d_image % elt) != 0) return fail(HEART_EINVAL, "image pointer misaligned");
    if (d_records && ((uintptr_t)d_records % 8) != 0) return fail(HEART_EINVAL, "records pointer misaligned");
    if (ray_offset + n_rays < ray_offset) return fail(HEART_EINVAL, "ray range overflows 64 bits");
    SourceParams P;
    char err[256] = {0};
    heart_status st = HEART_OK;
    std::vector<unsigned char> spectrum;
    if (prepared) P = *prepared;
    else st = build_source_params(src, &P, err, (int)sizeof err, &spectrum);
    if (st != HEART_OK) return fail(st, err);
    cudaStream_t cs = (cudaStream_t)stream;
    // a tabulated spectrum gets a stream-ordered device copy for this call
    struct FreeOnExit {
        void *p = nullptr;
        cudaStream_t s;
        ~FreeOnExit() { if (p) cudaFreeAsync(p, s); }
    } d_spec{nullptr, cs};
    cudaError_t e;
    if (!spectrum.empty()) {
        if ((e = cudaMallocAsync(&d_spec.p, spectrum.size(), cs)) != cudaSuccess) {
            d_spec.p = nullptr;
            return cuda_fail(e, "cudaMallocAsync spectrum");
        }
        // pageable source: staged before the call returns
        if ((e = cudaMemcpyAsync(d_spec.p, spectrum.data(), spectrum.size(), cudaMemcpyHostToDevice, cs)) != cudaSuccess)
            return cuda_fail(e, "spectrum upload");
        bind_spectrum(&P, d_spec.p);
    }
    e = cudaMemsetAsync(h->d_scratch, 0, kScratchWords * sizeof(unsigned long long), cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    void *img = d_image;
    if (!img) {
        // records only: count into the handle's own scratch image
        size_t bytes = (size_t)h->p.nx * h->p.ny * elt;
        if (!h->d_image_host_path || h->host_image_bytes < bytes) {
            if (h->d_image_host_path) cudaFree(h->d_image_host_path);
            h->d_image_host_path = nullptr;
            if ((e = cudaMalloc(&h->d_image_host_path, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc image");
            h->host_image_bytes = bytes;
        }
        img = h->d_image_host_path;
    }
    if (prec == HEART_FP64) {
        st = launch_fp64(h->p, P, n_rays, seed, ray_offset, img, h->d_scratch, (heart_ray_record *)d_records, cs, qe);
    } else if (takes_two_pass(h->p, P)) {
        // the two-pass trace runs on the device's shared hit queue (leased while enqueued);
        // records, when asked for, come from the same kernels
        WaveLease lease;
        st = wave_acquire(n_rays, cs, &lease);
        if (st != HEART_OK) return st;
        st = launch_fp32(h->p, P, n_rays, seed, ray_offset, img, h->d_scratch, cs, qe, lease.buf, lease.cap,
                         (heart_ray_record *)d_records);
        wave_release(lease, cs);
    } else if (d_records) {
        st = launch_fp32_records(h->p, P, n_rays, seed, ray_offset, img, h->d_scratch, (heart_ray_record *)d_records,
                                 cs, qe);
    } else {
        st = launch_fp32(h->p, P, n_rays, seed, ray_offset, img, h->d_scratch, cs, qe);
    }
    if (st != HEART_OK) return st;
    if (out || sync) {
        if ((e = cudaMemcpyAsync(h->h_scratch, h->d_scratch, kTallyN * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
            return cuda_fail(e, "tally copy");
        if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return cuda_fail(e, "trace");
        if (out) fill_tally(h->h_scratch, out);
        if (h->h_scratch[T_STUCK] > 0) return fail(HEART_ELIMIT, "a ray reached the collision cap");
    }
    return HEART_OK;
}

extern "C" heart_status heart_trace(heart_spectrometer *h, const heart_source_desc *src, uint64_t n_rays, uint64_t seed,
                                    uint64_t ray_offset, void *d_image, heart_precision precision, void *stream,
                                    heart_tally *out) {
    if (!d_image) return fail(HEART_EINVAL, "null image");
    return trace_impl(h, src, n_rays, seed, ray_offset, d_image, precision, nullptr, stream, out, false);
}

extern "C" heart_status heart_trace_records(heart_spectrometer *h, const heart_source_desc *src, uint64_t n_rays,
                                            uint64_t seed, uint64_t ray_offset, void *d_image,
                                            heart_precision precision, void *d_records, void *stream,
                                            heart_tally *out) {
    if (!d_records) return fail(HEART_EINVAL, "null records");
    // FP32 records come from the FP32 kernel's record variant
    return trace_impl(h, src, n_rays, seed, ray_offset, d_image, precision, d_records, stream, out, true);
}

extern "C" heart_status heart_trace_host(heart_spectrometer *h, const heart_source_desc *src, uint64_t n_rays,
                                         uint64_t seed, uint64_t ray_offset, void *h_image, heart_precision precision,
                                         heart_tally *out) {
    if (!h) return fail(HEART_EINVAL, "null spectrometer");
    if (!h_image) return fail(HEART_EINVAL, "null host image");
    size_t elt = h->p.count_type == HEART_COUNT_I64 ? 8 : 4;
    size_t bytes = (size_t)h->p.nx * h->p.ny * elt;
    cudaError_t e;
    if (!h->d_image_host_path || h->host_image_bytes < bytes) {
        if (h->d_image_host_path) cudaFree(h->d_image_host_path);
        h->d_image_host_path = nullptr;
        if ((e = cudaMalloc(&h->d_image_host_path, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc image");
        h->host_image_bytes = bytes;
    }
    cudaStream_t cs = 0;
    if ((e = cudaMemcpyAsync(h->d_image_host_path, h_image, bytes, cudaMemcpyHostToDevice, cs)) != cudaSuccess)
        return cuda_fail(e, "image upload");
    heart_status st = trace_impl(h, src, n_rays, seed, ray_offset, h->d_image_host_path, precision, nullptr, cs,
                                 nullptr, false);
    if (st != HEART_OK) return st;
    if ((e = cudaMemcpyAsync(h->h_scratch, h->d_scratch, kTallyN * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
        return cuda_fail(e, "tally copy");
    if ((e = cudaMemcpyAsync(h_image, h->d_image_host_path, bytes, cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
        return cuda_fail(e, "image download");
    if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return cuda_fail(e, "trace");
    if (out) fill_tally(h->h_scratch, out);
    if (h->h_scratch[T_STUCK] > 0) return fail(HEART_ELIMIT, "a ray reached the collision cap");
    return HEART_OK;
}

extern "C" heart_status heart_trace_energy(heart_spectrometer *h, const heart_source_desc *src, uint64_t n_rays,
                                           uint64_t seed, uint64_t ray_offset, void *d_image,
                                           uint64_t *d_energy_image, const heart_qe_table *qe,
                                           heart_precision precision, void *stream, heart_tally *out) {
    if (!h) return fail(HEART_EINVAL, "null spectrometer");
    if (!d_energy_image || ((uintptr_t)d_energy_image % 8) != 0) return fail(HEART_EINVAL, "null or misaligned energy image");
    QeParams Q;
    char err[256] = {0};
    heart_status st = build_qe_params(qe, (unsigned long long *)d_energy_image, &Q, err, (int)sizeof err);
    if (st != HEART_OK) return fail(st, err);
    return trace_impl(h, src, n_rays, seed, ray_offset, d_image, precision, nullptr, stream, out, false, &Q);
}

// mean keV per pixel of a calibration trace: energy (1e-6 keV units) / counts,
// NaN where no photon landed
template <typename CountT>
__global__ void k_mean_energy(const CountT *counts, const unsigned long long *energy, double *mean, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const CountT c = counts[i];
        mean[i] = c > 0 ? (double)energy[i] * 1e-6 / (double)c : __longlong_as_double(0x7ff8000000000000LL);
    }
}

extern "C" heart_status heart_calibration_map(heart_spectrometer *h, const heart_source_desc *src, double min_keV,
                                              double max_keV, uint64_t n_rays, uint64_t seed,
                                              heart_precision precision, void *d_counts, uint64_t *d_energy_image,
                                              double *d_mean_keV, void *stream, heart_tally *out) {
    if (!h) return fail(HEART_EINVAL, "null spectrometer");
    if (!src) return fail(HEART_EINVAL, "null source");
    if (!(min_keV > 0) || !(max_keV > min_keV) || !std::isfinite(max_keV))
        return fail(HEART_EINVAL, "calibration range needs 0 < min_keV < max_keV");
    const size_t elt = h->p.count_type == HEART_COUNT_I64 ? 8 : 4;
    if (!d_counts || ((uintptr_t)d_counts % elt) != 0) return fail(HEART_EINVAL, "null or misaligned count image");
    if (!d_mean_keV || ((uintptr_t)d_mean_keV % 8) != 0) return fail(HEART_EINVAL, "null or misaligned mean image");
    // the source's geometry with one uniform component on [min_keV, max_keV] (Sec. 3)
    heart_source_desc cal = *src;
    heart_spectral_component uni;
    std::memset(&uni, 0, sizeof uni);
    uni.kind = HEART_SRC_UNIFORM;
    uni.lo_keV = min_keV;
    uni.hi_keV = max_keV;
    uni.weight = 1.0;
    cal.components = &uni;
    cal.n_components = 1;
    cal.table_keV = nullptr;
    cal.table_pdf = nullptr;
    cal.n_table = 0;
    heart_status st = heart_trace_energy(h, &cal, n_rays, seed, 0, d_counts, d_energy_image, nullptr, precision,
                                         stream, out);
    if (st != HEART_OK && st != HEART_ELIMIT) return st;
    const size_t n = (size_t)h->p.nx * (size_t)h->p.ny;
    const int threads = 256;
    const int blocks = (int)std::min<size_t>((n + threads - 1) / threads, (size_t)num_sms() * 8);
    cudaStream_t cs = (cudaStream_t)stream;
    if (h->p.count_type == HEART_COUNT_I64)
        k_mean_energy<long long><<<blocks, threads, 0, cs>>>((const long long *)d_counts,
                                                             (const unsigned long long *)d_energy_image, d_mean_keV, n);
    else
        k_mean_energy<int><<<blocks, threads, 0, cs>>>((const int *)d_counts,
                                                       (const unsigned long long *)d_energy_image, d_mean_keV, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "calibration map kernel");
    return st;
}

extern "C" heart_status heart_trace_rays(heart_spectrometer *h, const heart_ray_arrays *rays, uint64_t n_rays,
                                         uint64_t seed, uint64_t ray_offset, void *d_image,
                                         heart_precision precision, void *d_records, void *stream,
                                         heart_tally *out) {
    if (!h) return fail(HEART_EINVAL, "null spectrometer");
    if (!rays) return fail(HEART_EINVAL, "null ray arrays");
    if (n_rays == 0) {                       // nothing to read: empty arrays may be null
        if (out) std::memset(out, 0, sizeof *out);
        return HEART_OK;
    }
    SourceParams P;
    char err[256] = {0};
    heart_status st = build_ray_params(rays, &P, err, (int)sizeof err);
    if (st != HEART_OK) return fail(st, err);
    if (!d_image && !d_records) return fail(HEART_EINVAL, "null image");
    return trace_impl(h, nullptr, n_rays, seed, ray_offset, d_image, precision, d_records, stream, out,
                      d_records != nullptr, nullptr, &P);
}
