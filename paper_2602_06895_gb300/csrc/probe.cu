// probe.cu -- FP64-pipe probes of the device.
//
// The FP64 map kernels are bound by the FP64 pipe's issue rate, so their roofline needs that
// rate as measured on the device, not derived from nominal unit counts and clocks.  Two kinds of
// kernels serve this:
//   - issue loops: eight independent chains of DFMA (or DADD, DMUL) per thread over a grid that
//     fills every SM, timed by the caller with CUDA events; instructions per second =
//     8 x iterations x threads / time;
//   - function loops: one call of an FP64 function (division, square root, exp, log, ...) per
//     iteration with arguments spread over a stated range, next to a loop that calls nothing; a
//     profiler's FP64-pipe instruction counters of the two give the function's FP64-pipe
//     instructions per call, the conversion from the method's operation counts (per class) to
//     the pipe's work.
// Every loop runs a fixed number of iterations and ends; nothing waits on anything.
#include <cuda_runtime.h>

#include <string>

#include "ps_internal.h"

namespace ps {
namespace {

constexpr int kProbeThreads = 256;

template <int kOp>
__global__ void __launch_bounds__(kProbeThreads) k_fp64_issue(int iters, double* sink) {
    const int t = blockIdx.x * kProbeThreads + threadIdx.x;
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1.0 + 1e-3 * static_cast<double>((t + k) & 1023);
    const double b = 1.0 + 0x1p-30, c = 0x1p-40;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (kOp == PS_PROBE_DFMA) a[k] = fma(a[k], b, c);
            else if (kOp == PS_PROBE_DADD) a[k] = a[k] + c;
            else a[k] = a[k] * b;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    sink[t] = s;
}

// The argument range of each function probe: x runs from lo to hi across the threads and
// iterations of a launch (one DADD per iteration, the same in the empty loop).
struct Range {
    double lo, hi;
};

__device__ __forceinline__ Range probe_range(int kind) {
    switch (kind) {
        case PS_PROBE_DIV: return {0.5, 50.0};
        case PS_PROBE_SQRT: return {1e-2, 1e2};
        case PS_PROBE_RSQRT: return {1e-2, 1e2};
        case PS_PROBE_EXP: return {-20.0, 20.0};
        case PS_PROBE_EXPM1: return {-2.0, 2.0};
        case PS_PROBE_LOG: return {1e-3, 1e3};
        case PS_PROBE_LOG1P: return {-0.5, 10.0};
        case PS_PROBE_POW: return {1e-2, 1.0};
        case PS_PROBE_ATAN: return {-50.0, 50.0};
        case PS_PROBE_ATAN2: return {-1.0, 1.0};
        case PS_PROBE_TAN: return {-1.5, 1.5};
        case PS_PROBE_SIN:
        case PS_PROBE_COS: return {0.0, 6.283185307179586};
        case PS_PROBE_SINCOSPI: return {0.0, 2.0};
        default: return {0.0, 1.0};
    }
}

template <int kKind>
__global__ void __launch_bounds__(kProbeThreads) k_fp64_func(int iters, double* sink) {
    const int t = blockIdx.x * kProbeThreads + threadIdx.x;
    const int n = gridDim.x * kProbeThreads;
    const Range R = probe_range(kKind);
    const double step = (R.hi - R.lo) / (static_cast<double>(n) * iters);
    double x = R.lo + (R.hi - R.lo) * static_cast<double>(t) / n;
    double acc = 0.0;
    for (int i = 0; i < iters; ++i) {
        double v;
        switch (kKind) {
            case PS_PROBE_DIV: v = 1.0 / x; break;
            case PS_PROBE_SQRT: v = sqrt(x); break;
            case PS_PROBE_RSQRT: v = rsqrt(x); break;
            case PS_PROBE_EXP: v = exp(x); break;
            case PS_PROBE_EXPM1: v = expm1(x); break;
            case PS_PROBE_LOG: v = log(x); break;
            case PS_PROBE_LOG1P: v = log1p(x); break;
            case PS_PROBE_POW: v = pow(x, -1.1); break;
            case PS_PROBE_ATAN: v = atan(x); break;
            case PS_PROBE_ATAN2: v = atan2(x, 0.7); break;
            case PS_PROBE_TAN: v = tan(x); break;
            case PS_PROBE_SIN: v = sin(x); break;
            case PS_PROBE_COS: v = cos(x); break;
            case PS_PROBE_SINCOSPI: {
                double s, c;
                sincospi(x, &s, &c);
                v = s + c;  // the one extra DADD of this probe (a pair of results)
                break;
            }
            default: v = x; break;  // the empty loop
        }
        acc += v;
        x += step;
    }
    sink[t] = acc;
}

template <int K>
void launch_func(int blocks, int iters, double* sink, cudaStream_t s) {
    k_fp64_func<K><<<blocks, kProbeThreads, 0, s>>>(iters, sink);
}

}  // namespace
}  // namespace ps

extern "C" int ps_fp64_probe(int kind, int blocks, int iters, double* sink, void* stream) {
    using namespace ps;
    if (blocks < 1 || iters < 1 || sink == nullptr) return PS_ERR_INVALID_ARGUMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (kind) {
        case PS_PROBE_DFMA: k_fp64_issue<PS_PROBE_DFMA><<<blocks, kProbeThreads, 0, s>>>(iters, sink); break;
        case PS_PROBE_DADD: k_fp64_issue<PS_PROBE_DADD><<<blocks, kProbeThreads, 0, s>>>(iters, sink); break;
        case PS_PROBE_DMUL: k_fp64_issue<PS_PROBE_DMUL><<<blocks, kProbeThreads, 0, s>>>(iters, sink); break;
        case PS_PROBE_EMPTY: launch_func<PS_PROBE_EMPTY>(blocks, iters, sink, s); break;
        case PS_PROBE_DIV: launch_func<PS_PROBE_DIV>(blocks, iters, sink, s); break;
        case PS_PROBE_SQRT: launch_func<PS_PROBE_SQRT>(blocks, iters, sink, s); break;
        case PS_PROBE_RSQRT: launch_func<PS_PROBE_RSQRT>(blocks, iters, sink, s); break;
        case PS_PROBE_EXP: launch_func<PS_PROBE_EXP>(blocks, iters, sink, s); break;
        case PS_PROBE_EXPM1: launch_func<PS_PROBE_EXPM1>(blocks, iters, sink, s); break;
        case PS_PROBE_LOG: launch_func<PS_PROBE_LOG>(blocks, iters, sink, s); break;
        case PS_PROBE_LOG1P: launch_func<PS_PROBE_LOG1P>(blocks, iters, sink, s); break;
        case PS_PROBE_POW: launch_func<PS_PROBE_POW>(blocks, iters, sink, s); break;
        case PS_PROBE_ATAN: launch_func<PS_PROBE_ATAN>(blocks, iters, sink, s); break;
        case PS_PROBE_ATAN2: launch_func<PS_PROBE_ATAN2>(blocks, iters, sink, s); break;
        case PS_PROBE_TAN: launch_func<PS_PROBE_TAN>(blocks, iters, sink, s); break;
        case PS_PROBE_SIN: launch_func<PS_PROBE_SIN>(blocks, iters, sink, s); break;
        case PS_PROBE_COS: launch_func<PS_PROBE_COS>(blocks, iters, sink, s); break;
        case PS_PROBE_SINCOSPI: launch_func<PS_PROBE_SINCOSPI>(blocks, iters, sink, s); break;
        default: return PS_ERR_INVALID_ARGUMENT;
    }
    if (cudaGetLastError() != cudaSuccess) return PS_ERR_CUDA;
    ps::count_launches(1);
    return PS_OK;
}
