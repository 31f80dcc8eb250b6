// sput_microbench.cu -- measured throughput peaks of the units the transport
// kernel issues to (sm_103a): FP32 FMA, the MUFU (XU) functions lg2 / ex2 /
// rsqrt / sin, the integer multiply-xor mix of a Philox4x32-10 round, and L2
// reductions (int32, int64, fp64) into a tally-sized array.  These are the
// denominators of the transport kernel's issue roofline and of its landing
// tally's atomic fraction.  Every kernel keeps its work in registers except the
// reductions, uses independent dependency chains so that throughput, not
// latency, bounds it, and writes one value per thread only if an impossible
// condition holds, so that the compiler keeps the work.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "sput.h"
#include "sput_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// FP32 FMA: 8 chains x 16 per iteration = 128 FMA lane-ops per thread and iteration
__global__ void __launch_bounds__(kThreads) mb_ffma(float* sink, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1234.5f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One MUFU function per kernel instance: 8 chains x 4 per iteration = 32 MUFU
// lane-ops per thread and iteration; the FMA that keeps each chain's argument in
// range runs on the FMA pipe, whose rate is 8x the XU rate.
template <int kOp>
__device__ __forceinline__ float mufu(float x)
{
    float y;
    if (kOp == 0) asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else if (kOp == 1) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else if (kOp == 2) asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int kOp>
__global__ void __launch_bounds__(kThreads) mb_mufu(float* sink, int iters)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (kOp == 1 ? -0.5f : 2.0f) - 1e-4f * (float)((threadIdx.x + c) & 15);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                const float y = mufu<kOp>(x[c]);
                // lg2, rsqrt, sin: x stays in [2, 3); ex2: x = -2^x stays in [-1, -0.5)
                x[c] = kOp == 1 ? -y : fmaf(y, 0.5f, 2.0f);
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1234.5f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Philox4x32-10 blocks (the transport's generator, Salmon et al. SC'11): 4
// independent counters per thread and iteration, 10 rounds each.
__global__ void __launch_bounds__(kThreads) mb_philox(float* sink, int iters, uint32_t k0, uint32_t k1)
{
    uint32_t acc = 0u;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t c0 = tid, c1 = (uint32_t)i, c2 = (uint32_t)q, c3 = 7u;
            uint32_t a0 = k0, a1 = k1;
#pragma unroll
            for (int r = 0; r < 10; ++r) {
                if (r) {
                    a0 += 0x9E3779B9u;
                    a1 += 0xBB67AE85u;
                }
                const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
                const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
                c0 = hi1 ^ c1 ^ a0;
                c1 = lo1;
                c2 = hi0 ^ c3 ^ a1;
                c3 = lo0;
            }
            acc ^= c0 ^ c1 ^ c2 ^ c3;
        }
    }
    if (acc == 0x12345678u) sink[tid] = (float)acc;
}

// L2 reductions (the atomic result is unused, as in the landing tally) at
// pseudo-random slots of an array of n_slots elements.
template <int kType>
__global__ void __launch_bounds__(kThreads) mb_red(void* buf, int n_slots, int iters)
{
    uint32_t h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    for (int i = 0; i < iters; ++i) {
        h = h * 1664525u + 1013904223u;
        const uint32_t slot = (uint32_t)(((unsigned long long)(h >> 8) * (unsigned long long)n_slots) >> 24);
        if (kType == 0) atomicAdd(static_cast<unsigned int*>(buf) + slot, 1u);
        else if (kType == 1) atomicAdd(static_cast<unsigned long long*>(buf) + slot, 1ull);
        else atomicAdd(static_cast<double*>(buf) + slot, 1.0);
    }
}

sput_status mb_fail(sput_status s, const std::string& msg)
{
    sput::set_last_error(msg.c_str());
    return s;
}

}  // namespace

extern "C" {

sput_status sput_microbench(int device, int kind, int n_slots, void* scratch, size_t scratch_bytes, int iters,
                            void* stream, sput_microbench_result* out)
{
    if (!out || !scratch) return mb_fail(SPUT_ERR_INVALID_ARG, "NULL argument");
    if (kind < 0 || kind > SPUT_MB_RED_F64) return mb_fail(SPUT_ERR_INVALID_ARG, "unknown microbenchmark kind");
    if (iters < 1 || iters > (1 << 24)) return mb_fail(SPUT_ERR_INVALID_ARG, "iters must be in [1, 2^24]");
    const bool red = kind >= SPUT_MB_RED_I32;
    const size_t elem = kind == SPUT_MB_RED_I32 ? 4 : 8;
    if (red && (n_slots < 1 || n_slots > (1 << 24) || scratch_bytes < elem * (size_t)n_slots))
        return mb_fail(SPUT_ERR_INVALID_ARG, "reductions need 1 <= n_slots <= 2^24 and scratch >= n_slots elements");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
        return mb_fail(SPUT_ERR_CUDA, "cudaSetDevice failed");
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
    const int blocks_per_sm = 8;  // 64 warps per SM: every scheduler has 16 warps to pick from
    const int blocks = n_sm * blocks_per_sm;
    // the sink is written only under an impossible condition; it must still be a
    // valid address for blocks * threads floats
    if (!red && scratch_bytes < sizeof(float) * (size_t)blocks * kThreads) {
        cudaSetDevice(prev);
        return mb_fail(SPUT_ERR_INVALID_ARG, "scratch must hold SMs * 8 * 256 floats");
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float* sink = static_cast<float*>(scratch);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (red && e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, elem * (size_t)n_slots, s);
    double lane_ops_per_iter = 0.0;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // rep 0 warms up, rep 1 is timed
        if (rep == 1) e = cudaEventRecord(e0, s);
        switch (kind) {
        case SPUT_MB_FFMA: mb_ffma<<<blocks, kThreads, 0, s>>>(sink, iters, 0.999f, 0.001f); lane_ops_per_iter = 128; break;
        case SPUT_MB_MUFU_LG2: mb_mufu<0><<<blocks, kThreads, 0, s>>>(sink, iters); lane_ops_per_iter = 32; break;
        case SPUT_MB_MUFU_EX2: mb_mufu<1><<<blocks, kThreads, 0, s>>>(sink, iters); lane_ops_per_iter = 32; break;
        case SPUT_MB_MUFU_RSQ: mb_mufu<2><<<blocks, kThreads, 0, s>>>(sink, iters); lane_ops_per_iter = 32; break;
        case SPUT_MB_MUFU_SIN: mb_mufu<3><<<blocks, kThreads, 0, s>>>(sink, iters); lane_ops_per_iter = 32; break;
        case SPUT_MB_PHILOX: mb_philox<<<blocks, kThreads, 0, s>>>(sink, iters, 11u, 13u); lane_ops_per_iter = 4; break;
        case SPUT_MB_RED_I32: mb_red<0><<<blocks, kThreads, 0, s>>>(scratch, n_slots, iters); lane_ops_per_iter = 1; break;
        case SPUT_MB_RED_I64: mb_red<1><<<blocks, kThreads, 0, s>>>(scratch, n_slots, iters); lane_ops_per_iter = 1; break;
        default: mb_red<2><<<blocks, kThreads, 0, s>>>(scratch, n_slots, iters); lane_ops_per_iter = 1; break;
        }
        e = cudaGetLastError();
        if (rep == 1 && e == cudaSuccess) e = cudaEventRecord(e1, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return mb_fail(SPUT_ERR_CUDA, cudaGetErrorString(e));
    out->ops = lane_ops_per_iter * (double)iters * (double)blocks * (double)kThreads;
    out->ms = ms;
    out->ops_per_s = ms > 0.0f ? out->ops / (ms * 1e-3) : 0.0;
    out->blocks = blocks;
    out->threads = kThreads;
    return SPUT_OK;
}

}  // extern "C"
