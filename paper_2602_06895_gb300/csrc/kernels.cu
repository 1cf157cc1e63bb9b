// kernels.cu -- sm_103a kernels of the phase-space library.
//
// ps_map_kernel evaluates the compiled instruction list of a channel (the
// paper's compute graph, Sec. 3.1 / Fig. compute_graph) for one event per
// thread.  All instructions of an event run back to back in that thread: the
// values live in a per-thread slot file in shared memory (slot s of thread t at
// smem[s * block + t], conflict-free), the byte-code, immediates and VEGAS grid
// of the channel are staged in shared memory once per channel change, and only
// the declared outputs (SoA, coalesced) and one partial-sum record per tile of
// `block` events reach global memory.  Tiles of all channels are distributed
// over a persistent grid; tile -> channel is a scan of at most 32 prefix sums
// held in the kernel parameters.
//
// Every branch inside an op depends only on the op's immediates (warp-uniform)
// or is resolved by selects, so the warps of a channel never diverge.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "map_device.cuh"
#include "ps_internal.h"

namespace ps {

static unsigned long long g_launches = 0;


// The interpreter's policy: a channel change stages its byte-code, immediates and VEGAS grid in
// shared memory; an event runs the byte-code on the thread's column of the slot file.
template <bool kMix>
struct InterpPolicy {
    const LaunchParams& lp;
    dev::Frame f;
    int32_t* s_code;
    double* s_imm;
    float* s_immf;
    double* s_grid;
    int out_pc;
    __device__ __forceinline__ void stage(int c, const ChannelLaunch& C) {
        const int B = lp.block, tid = threadIdx.x;
        for (int i = tid; i < C.code_len; i += B) s_code[i] = lp.code[C.code_off + i];
        for (int i = tid; i < C.imm_len; i += B) s_imm[i] = lp.imm[C.imm_off + i];
        if (kMix)
            for (int i = tid; i < C.imm_len; i += B) s_immf[i] = static_cast<float>(lp.imm[C.imm_off + i]);
        double* g = s_grid + kTrigDoubles;  // the grid after the azimuth table
        if (kMix) {
            dev::stage_grid(reinterpret_cast<float*>(g), lp.grid + C.grid_off, C.vdims, C.vbins, tid, B);
        } else {
            dev::stage_trig(s_grid, tid, B);
            dev::stage_grid(g, lp.grid + C.grid_off, C.vdims, C.vbins, tid, B);
        }
        __syncthreads();
        out_pc = dev::find_output(s_code, C.code_len);
    }
    __device__ __forceinline__ double event(int c, const ChannelLaunch& C, int64_t ev, int64_t local, bool active) {
        dev::load_inputs<kMix>(f, lp, c, C.n_random, ev, local, active);
        double* g = s_grid + kTrigDoubles;
        if (kMix) dev::run_code_mixed(s_code, out_pc, f, reinterpret_cast<float*>(g), C.vbins, lp.status + 1, active);
        else dev::run_code(s_code, out_pc, f, g, C.vbins, lp.status + 1, active);
        return dev::store_outputs<kMix>(f, s_code + out_pc + 3, s_code[out_pc + 1], lp, C, local, active);
    }
};

template <bool kMix>
__global__ void __launch_bounds__(256) ps_map_kernel(const __grid_constant__ LaunchParams lp) {
    extern __shared__ __align__(16) double smem[];
    const int B = lp.block;
    double* s_imm = smem;
    double* s_grid = s_imm + lp.smem_imm;
    double* s_slots = s_grid + lp.smem_grid;
    double* s_red = s_slots + static_cast<size_t>(lp.smem_slots) * B;
    int32_t* s_code = reinterpret_cast<int32_t*>(s_red + 4 * (B / 32));
    float* s_immf = reinterpret_cast<float*>(s_code + lp.smem_code_ints);  // mixed mode: float immediates
    InterpPolicy<kMix> pol{lp, dev::Frame{s_slots + threadIdx.x, s_imm, B, s_immf}, s_code, s_imm, s_immf, s_grid, 0};
    dev::map_tiles(lp, pol, s_red);
}

// One CTA per channel sums the channel's tile partials in a fixed order (deterministic); in
// streaming mode the launch's sums are added to the statistics of the earlier launches. A step of
// 1e7 events has ~1e5 tiles: each thread keeps four loads in flight, since one CTA reading them
// one at a time waits on memory latency.
constexpr int kReduceThreads = 1024;
constexpr int kReduceUnroll = 4;

__global__ void __launch_bounds__(kReduceThreads) ps_reduce_kernel(const __grid_constant__ LaunchParams lp,
                                                                   double* stats) {
    const int c = blockIdx.x;
    const ChannelLaunch& C = lp.ch[c];
    const int64_t t0 = C.tile_begin;
    const int64_t t1 = (c + 1 < lp.n_ch) ? lp.ch[c + 1].tile_begin : lp.n_tiles;
    double a0[kReduceUnroll], a1[kReduceUnroll], a2[kReduceUnroll], a3[kReduceUnroll];
#pragma unroll
    for (int u = 0; u < kReduceUnroll; ++u) a0[u] = a1[u] = a2[u] = a3[u] = 0.0;
    const int64_t stride = kReduceThreads;
    for (int64_t t = t0 + threadIdx.x; t < t1; t += kReduceUnroll * stride) {
        double2 lo[kReduceUnroll], hi[kReduceUnroll];
#pragma unroll
        for (int u = 0; u < kReduceUnroll; ++u) {  // the loads first, then the sums
            const int64_t tu = t + u * stride;
            const double2* tp = reinterpret_cast<const double2*>(lp.tile_partials + 4 * tu);
            lo[u] = tu < t1 ? tp[0] : make_double2(0.0, 0.0);
            hi[u] = tu < t1 ? tp[1] : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < kReduceUnroll; ++u) {
            a0[u] += lo[u].x;
            a1[u] += lo[u].y;
            a2[u] += hi[u].x;
            a3[u] = fmax(a3[u], hi[u].y);
        }
    }
    double v0 = (a0[0] + a0[1]) + (a0[2] + a0[3]);
    double v1 = (a1[0] + a1[1]) + (a1[2] + a1[3]);
    double v2 = (a2[0] + a2[1]) + (a2[2] + a2[3]);
    double v3 = fmax(fmax(a3[0], a3[1]), fmax(a3[2], a3[3]));
    // a fixed tree: within each warp by shuffles, then across the warps in shared memory
    for (int s = 16; s > 0; s >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, s);
        v1 += __shfl_down_sync(0xffffffffu, v1, s);
        v2 += __shfl_down_sync(0xffffffffu, v2, s);
        v3 = fmax(v3, __shfl_down_sync(0xffffffffu, v3, s));
    }
    __shared__ double red[4][kReduceThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = v0;
        red[1][warp] = v1;
        red[2][warp] = v2;
        red[3][warp] = v3;
    }
    __syncthreads();
    if (warp != 0) return;
    v0 = red[0][lane];
    v1 = red[1][lane];
    v2 = red[2][lane];
    v3 = red[3][lane];
    for (int s = 16; s > 0; s >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, s);
        v1 += __shfl_down_sync(0xffffffffu, v1, s);
        v2 += __shfl_down_sync(0xffffffffu, v2, s);
        v3 = fmax(v3, __shfl_down_sync(0xffffffffu, v3, s));
    }
    if (lane == 0) {
        double* o = stats + 5 * c;
        if (lp.stats_mode && *lp.stats_mode != 0) {  // streaming: add this launch to the running sums
            o[0] += static_cast<double>(C.n_events);
            o[1] += v0;
            o[2] += v1;
            o[3] += v2;
            o[4] = fmax(o[4], v3);
        } else {
            o[0] = static_cast<double>(C.n_events);
            o[1] = v0;
            o[2] = v1;
            o[3] = v2;
            o[4] = v3;
        }
    }
}

// ---------------------------------------------------------------- VEGAS training histogram
// The importance sums of VEGAS training, sum of w^2 per (dimension, bin of the unmapped r), for
// every channel of a launch, added in a fixed order so that an adaptation is reproducible bit for
// bit and does not depend on how tiles were scheduled.  Chunk k of a channel is one CTA of the
// first kernel: kHistChunks equal slices of the channel's events, walked in event order in blocks
// of kHistThreads.  Each block stages w^2 (from the stored weights) and the bin of every mapped
// dimension (the event's random numbers, regenerated from Philox or read back), then thread t adds,
// in event order, the w^2 of the events that fall into its entries t, t + kHistThreads, ...  The
// second kernel adds a channel's chunks in chunk order into the histogram.
__global__ void __launch_bounds__(kHistThreads) ps_hist_partial_kernel(const __grid_constant__ LaunchParams lp,
                                                                         double* part, int stride) {
    const int c = blockIdx.y, k = blockIdx.x, tid = threadIdx.x;
    const ChannelLaunch& C = lp.ch[c];
    const int nb = C.vdims * C.vbins;
    if (nb == 0) return;
    __shared__ double s_w2[kHistThreads];
    __shared__ uint8_t s_bin[kHistMaxDims * kHistThreads];
    const int64_t len = (C.n_events + kHistChunks - 1) / kHistChunks;
    const int64_t e0 = min(C.n_events, k * len), e1 = min(C.n_events, e0 + len);
    double acc[kHistEntries];
#pragma unroll
    for (int i = 0; i < kHistEntries; ++i) acc[i] = 0.0;
    for (int64_t base = e0; base < e1; base += kHistThreads) {
        const int64_t e = base + tid;
        if (e < e1) {
            const double w = lp.w[C.col_off + e];
            s_w2[tid] = w * w;
            const int64_t ev = C.ev_offset + e;
            for (int j = 0; j < C.vdims; j += 2) {
                double r0, r1 = 0.5;
                if (lp.r != nullptr) {
                    r0 = lp.r[j * lp.ld_r + e];
                    if (j + 1 < C.vdims) r1 = lp.r[(j + 1) * lp.ld_r + e];
                } else {
                    const uint4 o = rng::philox4x32_10(make_uint4(static_cast<uint32_t>(ev), static_cast<uint32_t>(ev >> 32),
                                                             static_cast<uint32_t>(c), static_cast<uint32_t>(j >> 1)),
                                                  static_cast<uint32_t>(lp.seed), static_cast<uint32_t>(lp.seed >> 32));
                    r0 = rng::unit_from_bits(o.y, o.x);
                    r1 = rng::unit_from_bits(o.w, o.z);
                }
                s_bin[j * kHistThreads + tid] = static_cast<uint8_t>(min(max(static_cast<int>(r0 * C.vbins), 0), C.vbins - 1));
                if (j + 1 < C.vdims)
                    s_bin[(j + 1) * kHistThreads + tid] =
                        static_cast<uint8_t>(min(max(static_cast<int>(r1 * C.vbins), 0), C.vbins - 1));
            }
        }
        __syncthreads();
        const int n = static_cast<int>(min(static_cast<int64_t>(kHistThreads), e1 - base));
#pragma unroll
        for (int i = 0; i < kHistEntries; ++i) {
            const int idx = tid + i * kHistThreads;
            if (idx < nb) {
                const int j = idx / C.vbins, b = idx - j * C.vbins;
                const uint8_t* bins = s_bin + j * kHistThreads;
                double a = acc[i];
                for (int t = 0; t < n; ++t)
                    if (bins[t] == b) a += s_w2[t];
                acc[i] = a;
            }
        }
        __syncthreads();
    }
    double* o = part + (static_cast<int64_t>(c) * kHistChunks + k) * stride;
#pragma unroll
    for (int i = 0; i < kHistEntries; ++i) {
        const int idx = tid + i * kHistThreads;
        if (idx < nb) o[idx] = acc[i];
    }
}

__global__ void __launch_bounds__(kHistThreads) ps_hist_reduce_kernel(const __grid_constant__ LaunchParams lp,
                                                                        const double* part, int stride) {
    const int c = blockIdx.y;
    const ChannelLaunch& C = lp.ch[c];
    const int idx = blockIdx.x * kHistThreads + threadIdx.x;
    if (idx >= C.vdims * C.vbins) return;
    const double* q = part + static_cast<int64_t>(c) * kHistChunks * stride + idx;
    double s = 0.0;
    for (int k = 0; k < kHistChunks; ++k) s += q[static_cast<int64_t>(k) * stride];
    lp.hist[C.hist_off + idx] += s;
}

size_t smem_bytes_for(const LaunchParams& lp) {
    size_t doubles = static_cast<size_t>(lp.smem_imm) + lp.smem_grid + static_cast<size_t>(lp.smem_slots) * lp.block +
                     4 * (lp.block / 32);
    return doubles * sizeof(double) + static_cast<size_t>(lp.smem_code_ints) * sizeof(int32_t) +
           (lp.mixed ? static_cast<size_t>(lp.smem_imm) * sizeof(float) : 0);
}

static int cuda_fail(cudaError_t e, const char* what, std::string* err) {
    *err = std::string(what) + ": " + cudaGetErrorString(e);
    return PS_ERR_CUDA;
}

int max_ctas_per_sm(int block, size_t smem, int mixed, int* out, std::string* err) {
    const void* fn = mixed ? reinterpret_cast<const void*>(ps_map_kernel<true>)
                           : reinterpret_cast<const void*>(ps_map_kernel<false>);
    // The dynamic shared-memory limit is a per-kernel, per-device setting shared by every program:
    // it only ever grows, so a program created later with a smaller slot file cannot lower the
    // limit below what an earlier program launches with.
    static std::mutex mu;
    static int limit[kMaxDevices][2] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice", err);
    if (dev < 0 || dev >= kMaxDevices) {
        *err = "device index beyond the library's limit";
        return PS_ERR_INVALID_ARGUMENT;
    }
    {
        std::lock_guard<std::mutex> lock(mu);
        int& cur = limit[dev][mixed ? 1 : 0];
        if (static_cast<int>(smem) > cur) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute", err);
            cur = static_cast<int>(smem);
        }
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, block, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor", err);
    return PS_OK;
}

int launch_map(const LaunchParams& lp, int grid_ctas, size_t smem, void* stream, std::string* err) {
    if (lp.n_tiles == 0) return PS_OK;
    if (lp.mixed) ps_map_kernel<true><<<grid_ctas, lp.block, smem, static_cast<cudaStream_t>(stream)>>>(lp);
    else ps_map_kernel<false><<<grid_ctas, lp.block, smem, static_cast<cudaStream_t>(stream)>>>(lp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ps_map_kernel launch", err);
    __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
    return PS_OK;
}

int launch_reduce(const LaunchParams& lp, double* stats, void* stream, std::string* err) {
    ps_reduce_kernel<<<lp.n_ch, kReduceThreads, 0, static_cast<cudaStream_t>(stream)>>>(lp, stats);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ps_reduce_kernel launch", err);
    __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
    return PS_OK;
}

int launch_hist(const LaunchParams& lp, double* part, int stride, void* stream, std::string* err) {
    if (lp.hist == nullptr || stride <= 0) return PS_OK;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    ps_hist_partial_kernel<<<dim3(kHistChunks, lp.n_ch), kHistThreads, 0, cs>>>(lp, part, stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ps_hist_partial_kernel launch", err);
    ps_hist_reduce_kernel<<<dim3((stride + kHistThreads - 1) / kHistThreads, lp.n_ch), kHistThreads, 0, cs>>>(lp, part,
                                                                                                            stride);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ps_hist_reduce_kernel launch", err);
    __atomic_add_fetch(&g_launches, 2ULL, __ATOMIC_RELAXED);
    return PS_OK;
}

bool is_hist_kernel(const void* func) {
    return func == reinterpret_cast<const void*>(ps_hist_partial_kernel) ||
           func == reinterpret_cast<const void*>(ps_hist_reduce_kernel);
}

// Copies the statistics into host-mapped pinned memory: the read-back of ps_stats uses no copy
// engine, so it does not queue behind large device-to-host copies of event records.
__global__ void __launch_bounds__(256) ps_copy_kernel(double* dst, const double* src, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i];
}

int launch_copy(double* dst, const double* src, int n, void* stream, std::string* err) {
    if (n <= 0) return PS_OK;
    ps_copy_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(dst, src, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "ps_copy_kernel launch", err);
    __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED);
    return PS_OK;
}

unsigned long long launch_count() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
void count_launches(int n) { __atomic_add_fetch(&g_launches, static_cast<unsigned long long>(n), __ATOMIC_RELAXED); }
bool is_reduce_kernel(const void* func) { return func == reinterpret_cast<const void*>(ps_reduce_kernel); }

// ---------------------------------------------------------------- mixed-form helpers
// Elementwise application of one device helper of the map kernels (ps_mixed_helpers).
template <int kKind, class In, class Out>
__global__ void __launch_bounds__(256) ps_mixed_helper_kernel(const In* in, Out* out, int64_t n) {
    for (int64_t i = blockIdx.x * 256LL + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * 256) {
        if constexpr (kKind == PS_MIXED_F2D) out[i] = dev::mx::f2d(in[i]);
        else if constexpr (kKind == PS_MIXED_D2F) out[i] = dev::mx::d2f(in[i]);
        else if constexpr (kKind == PS_MIXED_SQRT64) out[i] = dev::mx::sqrt64(in[i]);
        else if constexpr (kKind == PS_MIXED_TAN_QUARTER) out[i] = dev::tan_quarter(in[i]);
        else out[i] = dev::mx::rcp64(in[i]);
    }
}

// The FP64 azimuth (ps_mixed_helpers, PS_MIXED_SINCOS_TURN): each CTA stages its table first.
__global__ void __launch_bounds__(256) ps_turn_kernel(const double* in, double* out, int64_t n) {
    __shared__ double t[kTrigDoubles];
    dev::stage_trig(t, threadIdx.x, 256);
    __syncthreads();
    for (int64_t i = blockIdx.x * 256LL + threadIdx.x; i < n; i += static_cast<int64_t>(gridDim.x) * 256) {
        double s, c;
        dev::sincos_turn(in[i], t, s, c);
        out[2 * i] = c;
        out[2 * i + 1] = s;
    }
}

// ---------------------------------------------------------------- allocation-free scratch
// Fixed scratch for ps_generate_noalloc: kNoallocTiles per-tile partial-sum records (4 doubles
// each, 4 MiB) in a file-scope device array.  Every device that loads the library holds it until
// the process exits.  Host code must not hand the symbol itself to a kernel (on the host it is
// only a stand-in); its device address is fetched once per device with cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[static_cast<size_t>(kNoallocTiles) * 4];

namespace {
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

int noalloc_scratch(int device, void** ptr, size_t* bytes, std::string* err) {
    if (device < 0 || device >= kMaxDevices) {
        *err = "device index beyond the library's limit";
        return PS_ERR_INVALID_ARGUMENT;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_ptr[device] == nullptr) {
        // set-up: the calling thread has `device` current (the caller guarantees it)
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)", err);
        g_noalloc_ptr[device] = p;
    }
    *ptr = g_noalloc_ptr[device];
    *bytes = sizeof(g_noalloc_scratch);
    return PS_OK;
}

}  // namespace ps

extern "C" int ps_mixed_helpers(int kind, const void* in, void* out, int64_t n, void* stream) {
    using namespace ps;
    if (n < 0 || (n > 0 && (in == nullptr || out == nullptr))) return PS_ERR_INVALID_ARGUMENT;
    if (kind < PS_MIXED_F2D || kind > PS_MIXED_TAN_QUARTER) return PS_ERR_INVALID_ARGUMENT;
    if (n == 0) return PS_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152LL * 16);
    const int g = static_cast<int>(blocks);
    switch (kind) {
        case PS_MIXED_F2D:
            ps_mixed_helper_kernel<PS_MIXED_F2D><<<g, 256, 0, s>>>(static_cast<const float*>(in), static_cast<double*>(out), n);
            break;
        case PS_MIXED_D2F:
            ps_mixed_helper_kernel<PS_MIXED_D2F><<<g, 256, 0, s>>>(static_cast<const double*>(in), static_cast<float*>(out), n);
            break;
        case PS_MIXED_SQRT64:
            ps_mixed_helper_kernel<PS_MIXED_SQRT64><<<g, 256, 0, s>>>(static_cast<const double*>(in), static_cast<double*>(out), n);
            break;
        case PS_MIXED_RCP64:
            ps_mixed_helper_kernel<PS_MIXED_RCP64><<<g, 256, 0, s>>>(static_cast<const double*>(in), static_cast<double*>(out), n);
            break;
        case PS_MIXED_TAN_QUARTER:
            ps_mixed_helper_kernel<PS_MIXED_TAN_QUARTER><<<g, 256, 0, s>>>(static_cast<const double*>(in), static_cast<double*>(out), n);
            break;
        default:
            ps_turn_kernel<<<g, 256, 0, s>>>(static_cast<const double*>(in), static_cast<double*>(out), n);
            break;
    }
    if (cudaGetLastError() != cudaSuccess) return PS_ERR_CUDA;
    count_launches(1);
    return PS_OK;
}
