// Measured integer-ALU throughput of the device: the denominator of the
// library's roofline report for the alignment kernels, which do int32
// add/max/compare/logic work rather than dense contractions.
//
// Every thread runs kChains independent dependency chains, each step of a
// chain being three int32 operations, so the instruction stream is limited by
// issue and ALU throughput, not by latency.  Two mixes are timed: add, max and
// xor (the wavefront and DP cell updates; 3 operations a step) and add, xor,
// shift and add (the extend's window arithmetic; 4 a step); the higher rate is
// the peak.  The grid fills every SM
// with 8 blocks of 256 threads (64 warps per SM).  The count is of
// source-level operations, the same unit the alignment
// kernels' work counters use; whatever the compiler makes of them here it can
// make of them there.
#include <cstdint>

#include "aim_internal.cuh"
#include "ranges.h"

namespace aim {
namespace {

constexpr int kChains = 8;
constexpr int kOpsPerStep[2] = {3, 4};   // source-level int32 ops per chain step of each mix

template <int MIX>
__global__ void __launch_bounds__(256) int_peak_kernel(int iters, int c1, int c2, int* sink) {
    int a[kChains], b[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        a[j] = (int)threadIdx.x * (j + 1) + c1;
        b[j] = (int)blockIdx.x + j * c2;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            if constexpr (MIX == 0) {
                a[j] = max(a[j] + c1, b[j]);                          // add, max
                b[j] = b[j] ^ a[j];                                    // xor
            } else {
                a[j] = (a[j] + c1) ^ b[j];                             // add, xor
                b[j] = b[j] + (int)((unsigned)a[j] << (c2 & 7));       // shift, add
            }
        }
    }
    int s = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j] ^ b[j];
    if (s == c2 * 7919 + 1) sink[blockIdx.x] = s;   // practically never true; keeps the chains alive
}

}  // namespace
}  // namespace aim

extern "C" int aim_measure_int_peak(int device, double* ops_per_s, double* kernel_ms, double* per_mix) {
    aim::Range range("aim_measure_int_peak");
    using namespace aim;
    if (!ops_per_s) return AIM_ERR_ARG;
    DeviceGuardImpl guard(device);
    if (!guard.ok) return AIM_ERR_CUDA;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return cuda_status(e);
    int* sink = nullptr;
    e = cudaMalloc(&sink, (size_t)sms * 8 * sizeof(int));
    if (e != cudaSuccess) return cuda_status(e);
    cudaStream_t st = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const unsigned blocks = (unsigned)sms * 8;
    const int iters = 1 << 16;
    double best_rate = 0.0, best_ms = 0.0;
    for (int mix = 0; mix < 2 && e == cudaSuccess; ++mix) {
        float best = 1e30f;
        // a warm-up launch, then the best of five timed launches (each about 10-20 ms)
        for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(t0, st);
            if (e == cudaSuccess) {
                if (mix == 0) int_peak_kernel<0><<<blocks, 256, 0, st>>>(iters, 3, 5, sink);
                else int_peak_kernel<1><<<blocks, 256, 0, st>>>(iters, 3, 5, sink);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaEventRecord(t1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
        }
        if (e != cudaSuccess) break;
        const double ops = (double)blocks * 256.0 * iters * kChains * kOpsPerStep[mix];
        const double rate = ops / (best * 1e-3);
        if (per_mix) per_mix[mix] = rate;
        if (rate > best_rate) { best_rate = rate; best_ms = best; }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_status(e);
    *ops_per_s = best_rate;
    if (kernel_ms) *kernel_ms = best_ms;
    return AIM_OK;
}
