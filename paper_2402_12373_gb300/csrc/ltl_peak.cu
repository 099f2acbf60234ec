// ltl_peak.cu -- throughput of the integer instructions the candidate
// kernels are made of.
//
// The log-step loops of F, G and U (Section 4) are 32-bit shifts and
// three-input bitwise operations; a candidate launch that is not held back by
// memory is bounded by how many of these the SMs retire per second.  This
// probe measures that rate on the device it runs on: every thread runs eight
// independent chains, each step of a chain being one shift and one
// three-input logic operation (x = x | (y & (x >> s))), so the rate is set by
// the integer pipes and not by latency.  The result is the roof that the
// per-candidate integer work is compared with.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ltl.h"
#include "ltl_internal.h"

namespace ltl {
namespace {

constexpr int kPeakChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 8;

__global__ void __launch_bounds__(kPeakThreads) int_peak_kernel(uint32_t *sink, uint32_t s, int iters) {
    uint32_t x[kPeakChains], y[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) {
        x[k] = threadIdx.x * 0x9E3779B9u + (uint32_t)k;
        y[k] = blockIdx.x * 0x85EBCA6Bu + (uint32_t)(7 * k + 1);
    }
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) {
            uint32_t t;
            asm volatile("shr.b32 %0, %1, %2;" : "=r"(t) : "r"(x[k]), "r"(s));
            // 0xF8 = a | (b & c) over the truth tables a = 0xF0, b = 0xCC, c = 0xAA
            asm volatile("lop3.b32 %0, %0, %1, %2, 0xF8;" : "+r"(x[k]) : "r"(y[k]), "r"(t));
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) acc ^= x[k] + y[k];
    if (acc == 0x9E3779B9u) sink[blockIdx.x] = acc;   // keeps every chain live
}

}  // namespace
}  // namespace ltl

using namespace ltl;

extern "C" {

ltl_status ltl_int32_peak(int iters, int repeats, double *ops_per_s, double *best_ms) {
    if (!ops_per_s || iters < 4 || repeats < 1) return fail(LTL_ERR_INVALID, "int32 peak: bad arguments");
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(LTL_ERR_CUDA, "int32 peak: no device");
    const int blocks = n_sm * kPeakCtasPerSm;
    uint32_t *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ltl_status rc = LTL_OK;
    float best = 0.f;
    if (cudaMalloc(&sink, sizeof(uint32_t) * blocks) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = fail(LTL_ERR_CUDA, "int32 peak: %s", cudaGetErrorString(cudaGetLastError()));
    } else {
        int_peak_kernel<<<blocks, kPeakThreads, 0, st>>>(sink, 3u, iters);   // warm-up
        if (cudaGetLastError() != cudaSuccess) rc = fail(LTL_ERR_CUDA, "int32 peak: launch failed");
        for (int r = 0; r < repeats && rc == LTL_OK; ++r) {
            cudaEventRecord(e0, st);
            int_peak_kernel<<<blocks, kPeakThreads, 0, st>>>(sink, 3u, iters);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = fail(LTL_ERR_CUDA, "int32 peak: %s", cudaGetErrorString(cudaGetLastError()));
            else if (r == 0 || ms < best)
                best = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    if (rc != LTL_OK) return rc;
    const double ops = 2.0 * kPeakChains * (double)iters * (double)blocks * kPeakThreads;
    *ops_per_s = ops / (best * 1e-3);
    if (best_ms) *best_ms = best;
    return LTL_OK;
}

}  // extern "C"
