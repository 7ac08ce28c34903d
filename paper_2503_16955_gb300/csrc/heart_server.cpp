// heart_server.cpp -- the request loop: continuous batching of trace jobs.
//
// Jobs are admitted in arrival order while their detector images fit under
// the memory cap; admitted jobs stay resident (tables in their spectrometer
// handles, images and tallies here) until released.  A worker thread plans
// rounds in arrival order: jobs with few rays left are traced whole, the
// others share a budget of rays per round oldest first, in long slices; slices
// of 2^18 rays or more run as single-job two-pass launches, the others
// together in one persistent batched launch.  Jobs that arrive
// while a round is on the GPU join the next round, which is enqueued before
// the previous one has finished (two rounds in flight), so the device never
// waits for the host.  Each ray keeps its counter-based stream
// (ray_offset = rays already traced for the job), and every FP32 kernel traces
// a ray bit for bit alike, so a job's image is the same whether it ran alone or
// mixed with others.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "heart_lib.h"

namespace heart {
namespace {

using Clock = std::chrono::steady_clock;

enum JobState { QUEUED = 0, ADMITTED = 1, DONE = 2, FAILED = 3 };

struct Job {
    uint64_t id = 0;
    heart_spectrometer *spec = nullptr;
    SourceParams P;
    std::vector<unsigned char> spectrum;     // tabulated spectrum, copied into d_block at admission
    uint64_t n = 0, seed = 0, scheduled = 0;
    heart_precision prec = HEART_FP32;
    size_t img_bytes = 0;
    void *d_block = nullptr;                 // image, then kTallyN tally words
    void *d_img = nullptr;
    unsigned long long *d_tally = nullptr;
    int state = QUEUED;
    int pending_rounds = 0;                  // rounds in flight that hold slices of this job
    heart_tally tally;
    heart_status status = HEART_OK;
    Clock::time_point t_submit, t_done;
};

struct Round {
    cudaEvent_t done = nullptr;
    void *dev = nullptr;                     // batch work plan block
    std::vector<unsigned char> host;         // its host image if no pinned buffer was large enough
    unsigned char *pin = nullptr;            // pinned host image of the block (asynchronous upload)
    size_t pin_cap = 0;
    std::vector<uint64_t> ids;               // jobs with a slice in this round
    std::vector<bool> last;                  // the slice was the job's final one
};

}  // namespace
}  // namespace heart

struct heart_server {
    size_t cap = 0, used = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t copy_stream = nullptr;      // tally read-back, never behind a queued round
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, heart::Job *> jobs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    uint64_t round_rays = 64ull << 20;       // rays per round for jobs beyond small_job (about 2.5 ms of GPU work)
    uint64_t min_slice = 1ull << 22;         // a large job's slice is never smaller (unless it is its last)
    uint64_t small_job = 1ull << 20;         // jobs with this many rays left are traced whole in a round
    uint64_t two_pass_min = 1ull << 18;      // slices this large run as two-pass launches, the rest batched
    // pinned host buffers for the rounds' work plans (reused; a round holds one until it retires)
    std::vector<std::pair<unsigned char *, size_t>> pins;
    unsigned long long *tally_pin = nullptr;          // pinned read-back of finished jobs' tallies
    size_t tally_pin_n = 0;
};

namespace heart {
namespace {

// a pinned host buffer of at least `bytes` from the server's free list (worker thread only)
void take_pin(heart_server *s, size_t bytes, unsigned char **p, size_t *cap) {
    for (size_t i = 0; i < s->pins.size(); ++i)
        if (s->pins[i].second >= bytes) {
            *p = s->pins[i].first;
            *cap = s->pins[i].second;
            s->pins.erase(s->pins.begin() + (long)i);
            return;
        }
    size_t want = 64 << 10;
    while (want < bytes) want <<= 1;
    void *h = nullptr;
    if (cudaHostAlloc(&h, want, cudaHostAllocDefault) != cudaSuccess) { *p = nullptr; *cap = 0; return; }
    *p = (unsigned char *)h;
    *cap = want;
}

void give_pin(heart_server *s, unsigned char *p, size_t cap) {
    if (p) s->pins.push_back({p, cap});
}

// admit queued jobs while their images fit (called with the lock held)
void admit(heart_server *s) {
    while (!s->queue.empty()) {
        Job *j = s->jobs[s->queue.front()];
        if (s->used + j->img_bytes > s->cap) break;
        // image, tallies, then the job's tabulated spectrum (if any)
        const size_t off_tally = (j->img_bytes + 15) & ~(size_t)15;
        const size_t off_spec = (off_tally + kTallyN * sizeof(unsigned long long) + 15) & ~(size_t)15;
        const size_t bytes = off_spec + j->spectrum.size();
        cudaError_t e = cudaMallocAsync(&j->d_block, bytes, s->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(j->d_block, 0, off_spec, s->stream);
        if (e == cudaSuccess && !j->spectrum.empty()) {
            e = cudaMemcpyAsync((char *)j->d_block + off_spec, j->spectrum.data(), j->spectrum.size(),
                                cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess) bind_spectrum(&j->P, (char *)j->d_block + off_spec);
        }
        s->queue.pop_front();
        if (e != cudaSuccess) {
            if (j->d_block) cudaFreeAsync(j->d_block, s->stream);
            j->d_block = nullptr;
            j->state = FAILED;
            j->status = HEART_ENOMEM;
            j->t_done = Clock::now();
            s->cv_done.notify_all();
            continue;
        }
        j->d_img = j->d_block;
        j->d_tally = (unsigned long long *)((char *)j->d_block + off_tally);
        s->used += j->img_bytes;
        j->state = ADMITTED;
    }
}

void finish_round(heart_server *s, Round &r) {
    cudaEventSynchronize(r.done);
    give_pin(s, r.pin, r.pin_cap);
    r.pin = nullptr;
    // the finished jobs' tallies: one asynchronous copy each into pinned memory, one wait
    std::vector<Job *> fin;
    std::unique_lock<std::mutex> lk(s->mu);
    for (size_t i = 0; i < r.ids.size(); ++i) {
        auto it = s->jobs.find(r.ids[i]);
        if (it == s->jobs.end()) continue;
        Job *j = it->second;
        --j->pending_rounds;
        if (r.last[i] && j->state == ADMITTED) fin.push_back(j);
    }
    lk.unlock();
    if (!fin.empty()) {
        if (s->tally_pin_n < fin.size()) {
            if (s->tally_pin) cudaFreeHost(s->tally_pin);
            s->tally_pin = nullptr;
            s->tally_pin_n = 0;
            size_t want = 64;
            while (want < fin.size()) want <<= 1;
            void *h = nullptr;
            if (cudaHostAlloc(&h, want * kTallyN * sizeof(unsigned long long), cudaHostAllocDefault) == cudaSuccess) {
                s->tally_pin = (unsigned long long *)h;
                s->tally_pin_n = want;
            }
        }
        std::vector<unsigned long long> pageable;
        unsigned long long *h = s->tally_pin;
        if (!h) {
            pageable.resize(fin.size() * kTallyN);
            h = pageable.data();
        }
        for (size_t i = 0; i < fin.size(); ++i)
            cudaMemcpyAsync(h + i * kTallyN, fin[i]->d_tally, kTallyN * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, s->copy_stream);
        cudaStreamSynchronize(s->copy_stream);
        lk.lock();
        const Clock::time_point now = Clock::now();
        for (size_t i = 0; i < fin.size(); ++i) {
            Job *j = fin[i];
            std::memcpy(&j->tally, h + i * kTallyN, sizeof(heart_tally));
            j->status = j->tally.stuck > 0 ? HEART_ELIMIT : HEART_OK;
            j->state = DONE;
            j->t_done = now;
        }
        lk.unlock();
    }
    cudaFreeAsync(r.dev, s->stream);
    cudaEventDestroy(r.done);
    r.dev = nullptr;
    s->cv_done.notify_all();
}

void worker_main(heart_server *s) {
    cudaSetDevice(s->device);
    std::deque<Round> inflight;
    for (;;) {
        std::vector<Job *> slice_jobs;
        std::vector<uint64_t> nr, seeds, offs;
        std::vector<bool> last;
        std::vector<Job *> fp64_jobs;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto has_work = [&] {
                if (s->stop) return true;
                admit(s);
                for (auto &kv : s->jobs)
                    if (kv.second->state == ADMITTED && kv.second->scheduled < kv.second->n) return true;
                return false;
            };
            if (inflight.empty()) s->cv_work.wait(lk, has_work);
            else has_work();
            if (s->stop && inflight.empty()) break;
            // plan the next round in arrival order: every job with at most small_job rays
            // left is traced whole (small jobs share one batched launch and never wait
            // behind large ones for more than a round); the round's budget of round_rays
            // goes to the other jobs oldest first, in slices of at least min_slice, so a
            // large job runs in a few long launches as it would alone
            std::vector<Job *> active;
            for (auto &kv : s->jobs)
                if (kv.second->state == ADMITTED && kv.second->scheduled < kv.second->n) active.push_back(kv.second);
            std::sort(active.begin(), active.end(), [](Job *a, Job *b) { return a->id < b->id; });
            uint64_t budget = s->round_rays;
            for (Job *j : active) {
                const uint64_t left = j->n - j->scheduled;
                uint64_t take = 0;
                if (left <= s->small_job) {
                    take = left;
                } else if (budget > 0) {
                    take = std::min<uint64_t>(left, std::max<uint64_t>(budget, s->min_slice));
                    budget -= std::min(budget, take);
                } else {
                    continue;
                }
                if (j->prec == HEART_FP64) { fp64_jobs.push_back(j); continue; }
                slice_jobs.push_back(j);
                nr.push_back(take);
                seeds.push_back(j->seed);
                offs.push_back(j->scheduled);
                j->scheduled += take;
                last.push_back(j->scheduled == j->n);
                ++j->pending_rounds;
            }
            for (Job *j : fp64_jobs) {
                // FP64 jobs run whole, with the plain kernel, in the same stream order
                nr.push_back(0);
                j->scheduled = j->n;
                ++j->pending_rounds;
            }
        }
        if (!slice_jobs.empty() || !fp64_jobs.empty()) {
            Round r;
            std::vector<const SpecParams *> S;
            std::vector<SourceParams> P;
            std::vector<void *> imgs;
            std::vector<unsigned long long *> tl;
            for (Job *j : slice_jobs) {
                S.push_back(&j->spec->p);
                P.push_back(j->P);
                imgs.push_back(j->d_img);
                tl.push_back(j->d_tally);
                r.ids.push_back(j->id);
            }
            r.last = last;
            heart_status st = HEART_OK;
            // Slices of 2^18 rays or more that the two-pass trace takes run as single-job
            // two-pass launches, the others share one persistent batched launch.  Every
            // FP32 kernel traces a ray bit for bit alike, so a job's image does not depend
            // on how the rounds slice it or which kernel a slice runs on.
            std::vector<const SpecParams *> bS;
            std::vector<SourceParams> bP;
            std::vector<void *> bimg;
            std::vector<unsigned long long *> btl;
            std::vector<uint64_t> bnr, bseed, boff;
            for (size_t i = 0; i < slice_jobs.size() && st == HEART_OK; ++i) {
                const SpecParams &sp = *S[i];
                if (nr[i] >= s->two_pass_min && takes_two_pass(sp, P[i])) {
                    WaveLease lease;
                    st = wave_acquire(nr[i], s->stream, &lease);
                    if (st != HEART_OK) break;
                    st = launch_fp32(sp, P[i], nr[i], seeds[i], offs[i], imgs[i], tl[i], s->stream, nullptr,
                                     lease.buf, lease.cap);
                    wave_release(lease, s->stream);
                } else {
                    bS.push_back(S[i]); bP.push_back(P[i]); bimg.push_back(imgs[i]); btl.push_back(tl[i]);
                    bnr.push_back(nr[i]); bseed.push_back(seeds[i]); boff.push_back(offs[i]);
                }
            }
            if (st == HEART_OK && !bS.empty()) {
                const size_t bytes = batch_bytes((int)bS.size());
                if (cudaMallocAsync(&r.dev, bytes, s->stream) != cudaSuccess) st = HEART_ENOMEM;
                unsigned long long *unused = nullptr;
                take_pin(s, bytes, &r.pin, &r.pin_cap);
                if (st == HEART_OK)
                    st = launch_batch(bS.data(), bP.data(), bnr.data(), bseed.data(), boff.data(), bimg.data(),
                                      (int)bS.size(), r.dev, r.host, s->stream, &unused, btl.data(), nullptr, r.pin,
                                      r.pin_cap);
            }
            for (Job *j : fp64_jobs) {
                heart_status s2 = launch_fp64(j->spec->p, j->P, j->n, j->seed, 0, j->d_img, j->d_tally, nullptr,
                                              s->stream);
                if (s2 != HEART_OK) st = s2;
                r.ids.push_back(j->id);
                r.last.push_back(true);
            }
            cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming);
            cudaEventRecord(r.done, s->stream);
            if (st != HEART_OK) {
                std::lock_guard<std::mutex> lk(s->mu);
                for (uint64_t id : r.ids) {
                    auto it = s->jobs.find(id);
                    if (it != s->jobs.end()) { it->second->state = FAILED; it->second->status = st; it->second->t_done = Clock::now(); }
                }
            }
            inflight.push_back(std::move(r));
        }
        // keep at most two rounds in flight; retire the oldest when full or idle
        while (inflight.size() >= 2 || (!inflight.empty() && slice_jobs.empty() && fp64_jobs.empty())) {
            finish_round(s, inflight.front());
            inflight.pop_front();
        }
    }
}

}  // namespace
}  // namespace heart

using namespace heart;

extern "C" heart_status heart_server_create(size_t mem_cap_bytes, heart_server **out) {
    if (!out) return fail(HEART_EINVAL, "null output pointer");
    *out = nullptr;
    if (mem_cap_bytes == 0) return fail(HEART_EINVAL, "memory cap must be > 0");
    heart_server *s = new (std::nothrow) heart_server();
    if (!s) return fail(HEART_ENOMEM, "host allocation failed");
    s->cap = mem_cap_bytes;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete s; return cuda_fail(e, "server stream"); }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return HEART_OK;
}

extern "C" heart_status heart_server_destroy(heart_server *s) {
    if (!s) return fail(HEART_EINVAL, "null server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
    cudaStreamSynchronize(s->stream);
    for (auto &kv : s->jobs) {
        if (kv.second->d_block) cudaFree(kv.second->d_block);
        delete kv.second;
    }
    for (auto &pb : s->pins) cudaFreeHost(pb.first);
    if (s->tally_pin) cudaFreeHost(s->tally_pin);
    cudaStreamDestroy(s->stream);
    cudaStreamDestroy(s->copy_stream);
    delete s;
    return HEART_OK;
}

extern "C" heart_status heart_submit(heart_server *s, heart_spectrometer *spec, const heart_source_desc *src,
                                     uint64_t n_rays, uint64_t seed, heart_precision precision, uint64_t *job_id) {
    if (!s || !spec || !job_id) return fail(HEART_EINVAL, "null argument");
    if (precision != HEART_FP32 && precision != HEART_FP64) return fail(HEART_EINVAL, "unknown precision");
    Job *j = new (std::nothrow) Job();
    if (!j) return fail(HEART_ENOMEM, "host allocation failed");
    char err[256] = {0};
    heart_status st = build_source_params(src, &j->P, err, (int)sizeof err, &j->spectrum);
    if (st != HEART_OK) { delete j; return fail(st, err); }
    const size_t elt = spec->p.count_type == HEART_COUNT_I64 ? 8 : 4;
    j->img_bytes = (size_t)spec->p.nx * spec->p.ny * elt;
    if (j->img_bytes > s->cap) { delete j; return fail(HEART_ENOMEM, "job image exceeds the memory cap"); }
    j->spec = spec;
    j->n = n_rays;
    j->seed = seed;
    j->prec = precision;
    std::memset(&j->tally, 0, sizeof j->tally);
    j->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        j->id = s->next_id++;
        s->jobs[j->id] = j;
        s->queue.push_back(j->id);
        *job_id = j->id;
    }
    s->cv_work.notify_all();
    return HEART_OK;
}

extern "C" heart_status heart_poll(heart_server *s, uint64_t job_id, int32_t timeout_ms, heart_tally *out,
                                   const void **d_image_out) {
    if (!s) return fail(HEART_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(HEART_ENOTFOUND, "unknown job id");
    Job *j = it->second;
    auto done = [&] { return j->state == DONE || j->state == FAILED; };
    if (!done()) {
        if (timeout_ms <= 0) return fail(HEART_EBUSY, "job not finished");
        if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
            return fail(HEART_ETIMEOUT, "job not finished within the timeout");
    }
    if (j->state == FAILED) return fail(j->status, "job failed");
    if (out) *out = j->tally;
    if (d_image_out) *d_image_out = j->d_img;
    if (j->status == HEART_ELIMIT) return fail(HEART_ELIMIT, "a ray reached the collision cap");
    return HEART_OK;
}

extern "C" heart_status heart_release(heart_server *s, uint64_t job_id) {
    if (!s) return fail(HEART_EINVAL, "null server");
    Job *j = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return fail(HEART_ENOTFOUND, "unknown job id");
        j = it->second;
        if (j->state != DONE && j->state != FAILED) return fail(HEART_EBUSY, "job still running");
        s->jobs.erase(it);
        if (j->d_block) s->used -= j->img_bytes;
    }
    if (j->d_block) cudaFreeAsync(j->d_block, s->stream);
    delete j;
    s->cv_work.notify_all();
    return HEART_OK;
}

extern "C" heart_status heart_job_latency(heart_server *s, uint64_t job_id, double *seconds) {
    if (!s || !seconds) return fail(HEART_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return fail(HEART_ENOTFOUND, "unknown job id");
    Job *j = it->second;
    if (j->state != DONE && j->state != FAILED) return fail(HEART_EBUSY, "job not finished");
    *seconds = std::chrono::duration<double>(j->t_done - j->t_submit).count();
    return HEART_OK;
}

extern "C" heart_status heart_fetch_image(heart_server *s, uint64_t job_id, void *dst, int32_t dst_is_host) {
    if (!s || !dst) return fail(HEART_EINVAL, "null argument");
    void *src = nullptr;
    size_t bytes = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return fail(HEART_ENOTFOUND, "unknown job id");
        Job *j = it->second;
        if (j->state != DONE) return fail(j->state == FAILED ? j->status : HEART_EBUSY, "job not finished");
        src = j->d_img;
        bytes = j->img_bytes;
    }
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, dst_is_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                    s->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->copy_stream);
    if (e != cudaSuccess) return cuda_fail(e, "image copy");
    return HEART_OK;
}
