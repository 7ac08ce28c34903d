// heart_lib.h -- library-internal declarations (handles, launchers).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "heart.h"
#include "heart_internal.h"

struct heart_spectrometer;
namespace heart {
// device scratch words per handle: tallies, then work counters of the
// persistent kernels
constexpr int kScratchWords = 64;
constexpr int kCounterWord = 32;     // first work-counter word

struct TuneConfig {
    int refill = 8;                    // pop new rays when this many lanes of a warp are idle
    uint32_t chunk_rays = 1u << 16;    // largest work item (rays) claimed by a block
    // register budget: 6 (80 registers) or 5 (96 registers); 5 is what the autotuner picked on
    // every benchmark run (the all-persistent 64-job batch: 1.25e10 rays/s against 8.8e9 at 6)
    int blocks_per_sm = 5;
};
extern TuneConfig g_tune;

extern thread_local std::string g_last_error;
heart_status fail(heart_status st, const char *msg);
heart_status cuda_fail(cudaError_t e, const char *what);
int num_sms();

// qe may be nullptr (no energy image)
heart_status launch_fp64(const SpecParams &S, const SourceParams &P, uint64_t n, uint64_t seed, uint64_t offset,
                         void *img, unsigned long long *tally, heart_ray_record *rec, cudaStream_t st,
                         const QeParams *qe = nullptr);
// queue of prepared hits for the two-pass FP32 trace: two buffers of `cap`
// rays each (a power of two from 2^20 to 2^26; consecutive chunks alternate
// between them so that a chunk's spawn pass can overlap the previous chunk's
// walk), one record per hit (96 bytes, 112 for a polarised source), then 2
// counters per chunk for kWaveGroup chunks
constexpr uint32_t kWaveMinCap = 1u << 20, kWaveMaxCap = 1u << 26;
constexpr int kWaveGroup = 1024;
// jobs of at least this many rays (one reflection order) run on the two-pass
// trace in batches and in the request loop, as single traces do
constexpr uint64_t kTwoPassMinRays = 1ull << 18;

// the two-pass trace takes every FP32 image trace but user rays with several
// reflection orders (those run on the persistent extended kernel)
inline bool takes_two_pass(const SpecParams &S, const SourceParams &P) { return !(P.user && S.n_orders > 1); }
constexpr int kWaveRec16 = 6;                  // 16-byte words per queued hit (a 96-byte record)
constexpr int kWaveRecMax16 = 7;               // with the polarisation word
inline size_t wave_buffer_bytes(uint32_t cap) { return (size_t)16 * kWaveRecMax16 * cap; }
inline size_t wave_bytes(uint32_t cap) { return 2 * wave_buffer_bytes(cap) + (size_t)2 * 8 * kWaveGroup; }
inline uint32_t wave_cap_for(uint64_t n) {
    uint32_t c = kWaveMinCap;
    while (c < kWaveMaxCap && (uint64_t)c < n) c <<= 1;
    return c;
}
struct WaveBuf {
    void *base;
    uint32_t cap, pad;
};
// wave / wave_cap: a leased hit queue (nullptr: the one-pass persistent kernel)
// rec (two-pass trace only): one heart_ray_record per ray, or nullptr
heart_status launch_fp32(const SpecParams &S, const SourceParams &P, uint64_t n, uint64_t seed, uint64_t offset,
                         void *img, unsigned long long *scratch, cudaStream_t st, const QeParams *qe = nullptr,
                         void *wave = nullptr, uint32_t wave_cap = 0, heart_ray_record *rec = nullptr);
// The hit queue of the two-pass FP32 trace: one per device, shared by every
// spectrometer handle, grown to the largest chunk asked for (never shrunk).
// wave_acquire locks it for the calling host thread while a trace is enqueued
// and makes the stream wait (on the GPU) for the queue's previous user;
// wave_release records the stream's position as the next user's start and
// unlocks.  Traces that need the queue therefore run one after another on the
// GPU whatever their streams; everything else stays concurrent.
struct WaveLease {
    void *buf;
    uint32_t cap;
    int device;
};
heart_status wave_acquire(uint64_t n, cudaStream_t st, WaveLease *out);
void wave_release(const WaveLease &lease, cudaStream_t st);
heart_status launch_fp32_records(const SpecParams &S, const SourceParams &P, uint64_t n, uint64_t seed,
                                 uint64_t offset, void *img, unsigned long long *scratch, heart_ray_record *rec,
                                 cudaStream_t st, const QeParams *qe = nullptr);
size_t batch_bytes(int n);
// device bytes of the jobs' tabulated spectra appended after the batch block
size_t spectra_bytes(const std::vector<unsigned char> *spectra, int n);
heart_status launch_batch(const SpecParams *const *S, const SourceParams *P, const uint64_t *n_rays,
                          const uint64_t *seeds, const uint64_t *offsets, void *const *imgs, int n, void *dev,
                          std::vector<unsigned char> &host, cudaStream_t st, unsigned long long **tallies_dev,
                          unsigned long long *const *tally_ptrs,
                          const std::vector<unsigned char> *spectra = nullptr, unsigned char *pinned = nullptr,
                          size_t pinned_cap = 0);
}  // namespace heart

struct heart_spectrometer {
    heart::SpecParams p;
    heart_spectrometer_desc desc;
    int device = 0;
    void *d_block = nullptr;              // tables + scratch, one allocation
    double *d_tab64 = nullptr;
    float *d_tab32 = nullptr;
    unsigned long long *d_scratch = nullptr;
    unsigned long long *h_scratch = nullptr;   // pinned tally copy
    void *d_image_host_path = nullptr;    // image buffer of heart_trace_host
    size_t host_image_bytes = 0;
};
