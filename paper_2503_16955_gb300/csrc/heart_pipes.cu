// heart_pipes.cu -- issue-rate microbenchmark of the SM pipes the ray path
// runs on (FP32 FMA, integer ALU and multiply, the SFU / MUFU, FP64), so that
// the kernels' per-pipe instruction counts can be stated as a fraction of what
// each pipe sustains on this GPU at the clocks it runs at.
//
// Each kernel runs eight chains of one instruction per thread (inline PTX, so
// the instruction is the one named, not the compiler's choice): chain j takes
// its own previous value, chain j + 1's, and for three-operand forms a
// loop-invariant register, so that operands come from different register
// banks or the operand-reuse cache.  32 warps per SM.  CUDA events give the
// whole-GPU rate per second; each block times its loop with clock64() (SM
// cycles) and %globaltimer (ns), whose ratio is the SM clock the run saw, and
// the rate per SM per clock is the rate per second over SMs x that clock.
// Loop overhead is one add, one compare and one branch per 64 measured
// instructions.
#include <cuda_runtime.h>

#include <cstring>

#include "heart.h"
#include "heart_lib.h"

namespace heart {
namespace {

constexpr int kPipeThreads = 256, kPipeBlocksPerSm = 4, kPipeUnroll = 8;

// one step of eight chains: r[j] = op(r[j], r[j + 1], c) (indices mod 8)
template <int OP>
__device__ __forceinline__ void pipe_step(uint32_t r[8], uint32_t c) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t &a = r[j];
        const uint32_t b = r[(j + 1) & 7];
        if (OP == HEART_PIPE_FFMA) {
            asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+r"(a) : "r"(b), "r"(c));
        } else if (OP == HEART_PIPE_LOP3) {
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a) : "r"(b), "r"(c));
        } else if (OP == HEART_PIPE_IADD3) {
            asm volatile("add.u32 %0, %0, %1;" : "+r"(a) : "r"(b));
        } else if (OP == HEART_PIPE_IMAD) {
            asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a) : "r"(b), "r"(c));
        } else if (OP == HEART_PIPE_IMAD_HI) {
            asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(a) : "r"(b));
        } else if (OP == HEART_PIPE_IMAD_WIDE) {
            // 32 x 32 -> 64 bits; the chain keeps the high half
            asm volatile("{\n\t.reg .u64 t;\n\t.reg .u32 lo;\n\tmul.wide.u32 t, %0, %1;\n\tmov.b64 {lo, %0}, t;\n\t}"
                         : "+r"(a) : "r"(b));
        } else if (OP == HEART_PIPE_MUFU_RSQ) {
            asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+r"(a));
        } else if (OP == HEART_PIPE_MUFU_EX2) {
            asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+r"(a));
        } else if (OP == HEART_PIPE_MUFU_LG2) {
            asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+r"(a));
        }
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// cycles[0]: summed clock64 cycles of the blocks' loops, cycles[1]: summed globaltimer ns
template <int OP>
__global__ void __launch_bounds__(kPipeThreads) k_pipe(uint32_t *sink, int iters, uint32_t seed,
                                                        unsigned long long *cycles) {
    uint32_t r[8];
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = 0x3f800000u + ((seed + t * 8u + (uint32_t)j) & 0xFFFFu);
    const uint32_t c = 0x3f800001u + (seed & 0xFFu);
    __syncthreads();
    const long long t0 = clock64();
    const unsigned long long g0 = global_ns();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPipeUnroll; ++u) pipe_step<OP>(r, c);
    }
    const long long t1 = clock64();
    const unsigned long long g1 = global_ns();
    uint32_t x = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) x ^= r[j];
    if (x == 0x9E3779B9u) sink[t] = x;                  // keeps the chains live; practically never taken
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(cycles, (unsigned long long)(t1 - t0));
        atomicAdd(cycles + 1, g1 - g0);
    }
}

// FP64 FMA chains (the plain path's pipe)
__global__ void __launch_bounds__(kPipeThreads) k_pipe_dfma(double *sink, int iters, uint32_t seed,
                                                            unsigned long long *cycles) {
    double r[8];
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int j = 0; j < 8; ++j) r[j] = 1.0 + 1e-9 * (double)((seed + t * 8u + (uint32_t)j) & 0xFFFFu);
    const double c = 1.0 + 1e-12 * (double)(seed & 0xFFu);
    __syncthreads();
    const long long t0 = clock64();
    const unsigned long long g0 = global_ns();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPipeUnroll; ++u) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(r[j]) : "d"(r[(j + 1) & 7]), "d"(c));
        }
    }
    const long long t1 = clock64();
    const unsigned long long g1 = global_ns();
    double x = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) x += r[j];
    if (x == 1.2345678) sink[t] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(cycles, (unsigned long long)(t1 - t0));
        atomicAdd(cycles + 1, g1 - g0);
    }
}

template <int OP>
cudaError_t run_pipe(int blocks, int iters, void *sink, unsigned long long *cyc, cudaStream_t st) {
    if constexpr (OP == HEART_PIPE_DFMA)
        k_pipe_dfma<<<blocks, kPipeThreads, 0, st>>>((double *)sink, iters, 12345u, cyc);
    else
        k_pipe<OP><<<blocks, kPipeThreads, 0, st>>>((uint32_t *)sink, iters, 12345u, cyc);
    return cudaGetLastError();
}

cudaError_t run_op(int op, int blocks, int iters, void *sink, unsigned long long *cyc, cudaStream_t st) {
    switch (op) {
    case HEART_PIPE_FFMA: return run_pipe<HEART_PIPE_FFMA>(blocks, iters, sink, cyc, st);
    case HEART_PIPE_LOP3: return run_pipe<HEART_PIPE_LOP3>(blocks, iters, sink, cyc, st);
    case HEART_PIPE_IADD3: return run_pipe<HEART_PIPE_IADD3>(blocks, iters, sink, cyc, st);
    case HEART_PIPE_IMAD: return run_pipe<HEART_PIPE_IMAD>(blocks, iters, sink, cyc, st);
    case HEART_PIPE_IMAD_HI: return run_pipe<HEART_PIPE_IMAD_HI>(blocks, iters, sink, cyc, st);
    case HEART_PIPE_IMAD_WIDE: return run_pipe<HEART_PIPE_IMAD_WIDE>(blocks, iters, sink, cyc, st);
    case HEART_PIPE_MUFU_RSQ: return run_pipe<HEART_PIPE_MUFU_RSQ>(blocks, iters, sink, cyc, st);
    case HEART_PIPE_MUFU_EX2: return run_pipe<HEART_PIPE_MUFU_EX2>(blocks, iters, sink, cyc, st);
    case HEART_PIPE_MUFU_LG2: return run_pipe<HEART_PIPE_MUFU_LG2>(blocks, iters, sink, cyc, st);
    default: return run_pipe<HEART_PIPE_DFMA>(blocks, iters, sink, cyc, st);
    }
}

}  // namespace
}  // namespace heart

using namespace heart;

extern "C" heart_status heart_pipe_peaks(void *stream, heart_pipe_rates *out) {
    if (!out) return fail(HEART_EINVAL, "heart_pipe_peaks: out is NULL");
    std::memset(out, 0, sizeof *out);
    cudaStream_t st = (cudaStream_t)stream;
    const int sms = num_sms();
    const int blocks = sms * kPipeBlocksPerSm;
    const size_t threads = (size_t)blocks * kPipeThreads;
    void *sink = nullptr;
    unsigned long long *cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, threads * sizeof(double) + 64);
    if (e != cudaSuccess) return cuda_fail(e, "heart_pipe_peaks: cudaMalloc");
    cyc = (unsigned long long *)((char *)sink + threads * sizeof(double));
    heart_status rc = HEART_OK;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        rc = cuda_fail(e, "heart_pipe_peaks: cudaEventCreate");
    }
    // loop trips per op: about 1-4 ms each at the expected rates (the same launch every
    // call, so that a profiler sees the timed configuration)
    static const int kIters[HEART_PIPE_NOPS] = {4096, 4096, 4096, 4096, 2048, 2048, 1024, 1024, 1024, 128};
    double clk_sum = 0.0;
    int clk_n = 0;
    for (int op = 0; op < HEART_PIPE_NOPS && rc == HEART_OK; ++op) {
        const int iters = kIters[op];
        float ms = 0.f;
        // one untimed warm-up launch, then the timed one
        for (int pass = 0; pass < 2 && rc == HEART_OK; ++pass) {
            if ((e = cudaMemsetAsync(cyc, 0, 16, st)) != cudaSuccess) { rc = cuda_fail(e, "memset"); break; }
            if ((e = cudaEventRecord(e0, st)) != cudaSuccess) { rc = cuda_fail(e, "event"); break; }
            if ((e = run_op(op, blocks, iters, sink, cyc, st)) != cudaSuccess) { rc = cuda_fail(e, "pipe kernel"); break; }
            if ((e = cudaEventRecord(e1, st)) != cudaSuccess) { rc = cuda_fail(e, "event"); break; }
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = cuda_fail(e, "pipe kernel"); break; }
            cudaEventElapsedTime(&ms, e0, e1);
        }
        if (rc != HEART_OK) break;
        unsigned long long acc[2] = {0, 0};
        if ((e = cudaMemcpy(acc, cyc, 16, cudaMemcpyDeviceToHost)) != cudaSuccess) {
            rc = cuda_fail(e, "heart_pipe_peaks: copy");
            break;
        }
        const double warp_inst = (double)threads / 32.0 * (double)iters * kPipeUnroll * 8.0;
        out->warp_inst_per_s[op] = warp_inst / (ms * 1e-3);
        // the SM clock of this run: clock64 cycles per globaltimer second, summed over the
        // blocks (a ratio within each block, whether or not all blocks run at once)
        const double clk = acc[1] > 0 ? (double)acc[0] / ((double)acc[1] * 1e-9) : 0.0;
        out->warp_inst_per_clk_sm[op] = clk > 0 ? out->warp_inst_per_s[op] / (clk * sms) : 0.0;
        if (clk > 0) {
            clk_sum += clk;
            ++clk_n;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    out->sms = sms;
    out->n_ops = HEART_PIPE_NOPS;
    out->sm_clock_hz = clk_n ? clk_sum / clk_n : 0.0;
    return rc;
}
