// unweight.cu -- event unweighting on the GPU (Sec. "Unweighting and file output").
//
// Maximum weight with a bounded over-weight share: w_max(eps) is the smallest t >= 0 with
//     sum_b max(0, w_b - t) <= eps * sum_b w_b.
// The excess is continuous and decreasing in t.  Non-negative doubles order like their bit
// patterns, so the root is located by a radix search over the bits of t: each pass splits the
// current bit range [lo, hi) into 256 buckets, histograms count and sum of the weights per
// bucket, and keeps the bucket in which the excess crosses eps S (the excess at a bucket's lower
// edge T follows from the counts and sums of all weights >= T).  The search stops when the kept
// bucket holds no weight (or is one bit pattern wide); then no weight lies strictly between the
// root and the bucket's upper edge, and w_max = (A - eps S) / K in closed form, A and K the sum
// and count of the weights above.  At most 8 passes (64 bits / 8 bits per pass).
//
// Every sum has a fixed order for a given batch size (per-block partials over a fixed grid,
// warp-private histograms filled in lane order by owner lanes, blocks combined in index order),
// so the result is reproducible bit for bit.
//
// Accept/reject: event b is kept iff u_b w_max < w_b, u_b the first uniform of the generator's
// Philox point of event (event_offset + b) in stream 0x556E7700; kept events carry max(w_b, w_max)
// and are written in increasing event order (per-block counts, one scan, per-block writes).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "philox.cuh"
#include "ps.h"

namespace ps {
void count_launches(int n);
namespace uw {

constexpr int kGrid = 512;          // blocks of the reductions and histograms (fixed: reproducible sums)
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBuckets = 256;
constexpr int kPasses = 8;
constexpr int kSelPerThread = 8;    // events per thread in the select kernels
constexpr int kSelBlock = kThreads * kSelPerThread;
constexpr uint32_t kStream = 0x556E7700u;

struct State {
    unsigned long long lo, hi;          // current bit range of the root, [lo, hi)
    double S, target, wmax;
    double carry_sum;                   // sum and count of the weights >= hi
    unsigned long long carry_cnt;
    unsigned long long invalid;
    double t;                           // the result once done
    int done;
};

__device__ __forceinline__ bool valid(double w) { return w >= 0.0 && w <= 1.7976931348623157e308; }

// per-block partials of sum, max and the number of invalid (negative or non-finite) weights
__global__ void __launch_bounds__(kThreads) k_partials(const double* w, int64_t n, double* part) {
    __shared__ double ss[kThreads], sm[kThreads];
    __shared__ unsigned long long si[kThreads];
    const int64_t chunk = (n + kGrid - 1) / kGrid;
    const int64_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    double s = 0.0, m = 0.0;
    unsigned long long bad = 0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += kThreads) {
        double v = w[i];
        if (valid(v)) {
            s += v;
            m = fmax(m, v);
        } else {
            ++bad;
        }
    }
    ss[threadIdx.x] = s;
    sm[threadIdx.x] = m;
    si[threadIdx.x] = bad;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            ss[threadIdx.x] += ss[threadIdx.x + o];
            sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
            si[threadIdx.x] += si[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = ss[0];
        part[3 * blockIdx.x + 1] = sm[0];
        part[3 * blockIdx.x + 2] = static_cast<double>(si[0]);
    }
}

__global__ void k_init(const double* part, double eps, State* st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double S = 0.0, m = 0.0, bad = 0.0;
    for (int b = 0; b < kGrid; ++b) {
        S += part[3 * b];
        m = fmax(m, part[3 * b + 1]);
        bad += part[3 * b + 2];
    }
    State s{};
    s.S = S;
    s.wmax = m;
    s.invalid = static_cast<unsigned long long>(bad);
    s.target = eps * S;
    s.lo = 0;
    s.hi = static_cast<unsigned long long>(__double_as_longlong(m)) + 1;
    s.carry_sum = 0.0;
    s.carry_cnt = 0;
    s.done = 0;
    if (S == 0.0 || s.target >= S) {  // nothing to keep above: every weight is below w_max = 0
        s.t = 0.0;
        s.done = 1;
    } else if (!(eps > 0.0)) {
        s.t = m;
        s.done = 1;
    }
    *st = s;
}

// one radix pass: per-block histogram of count and sum over the 256 buckets of [lo, hi)
__global__ void __launch_bounds__(kThreads) k_hist(const double* w, int64_t n, const State* st, double* hsum,
                                                   unsigned int* hcnt) {
    __shared__ double ws[kWarps][kBuckets];
    __shared__ unsigned int wc[kWarps][kBuckets];
    if (st->done) return;
    const unsigned long long lo = st->lo, hi = st->hi;
    const unsigned long long step = (hi - lo + kBuckets - 1) / kBuckets;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = lane; j < kBuckets; j += 32) {
        ws[warp][j] = 0.0;
        wc[warp][j] = 0;
    }
    __syncwarp();
    const int64_t chunk = (n + kGrid - 1) / kGrid;
    const int64_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    for (int64_t base = b0 + warp * 32; base < b1; base += kThreads) {
        const int64_t i = base + lane;
        double v = 0.0;
        int bk = -1;
        if (i < b1) {
            v = w[i];
            if (valid(v)) {
                unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v));
                if (u >= lo && u < hi) bk = static_cast<int>((u - lo) / step);
            }
        }
        // lane order, each bucket updated only by its owner lane (bucket mod 32)
        for (int src = 0; src < 32; ++src) {
            const double sv = __shfl_sync(0xffffffffu, v, src);
            const int sb = __shfl_sync(0xffffffffu, bk, src);
            if (sb >= 0 && (sb & 31) == lane) {
                ws[warp][sb] += sv;
                wc[warp][sb] += 1;
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kBuckets; j += kThreads) {
        double s = 0.0;
        unsigned int c = 0;
        for (int k = 0; k < kWarps; ++k) {
            s += ws[k][j];
            c += wc[k][j];
        }
        hsum[blockIdx.x * kBuckets + j] = s;
        hcnt[blockIdx.x * kBuckets + j] = c;
    }
}

// combine the block histograms in block order and choose the bucket holding the root
__global__ void __launch_bounds__(kBuckets) k_decide(const double* hsum, const unsigned int* hcnt, State* st) {
    __shared__ double bs[kBuckets];
    __shared__ unsigned long long bc[kBuckets];
    if (st->done) return;
    const int j = threadIdx.x;
    double s = 0.0;
    unsigned long long c = 0;
    for (int b = 0; b < kGrid; ++b) {
        s += hsum[b * kBuckets + j];
        c += hcnt[b * kBuckets + j];
    }
    bs[j] = s;
    bc[j] = c;
    __syncthreads();
    if (j != 0) return;
    State x = *st;
    const unsigned long long step = (x.hi - x.lo + kBuckets - 1) / kBuckets;
    double cum_s = x.carry_sum;
    unsigned long long cum_c = x.carry_cnt;
    int sel = 0;
    for (int k = kBuckets - 1; k >= 0; --k) {
        const unsigned long long edge = x.lo + static_cast<unsigned long long>(k) * step;
        if (edge >= x.hi) continue;
        cum_s += bs[k];
        cum_c += bc[k];
        const double T = __longlong_as_double(static_cast<long long>(edge));
        if (cum_s - T * static_cast<double>(cum_c) > x.target) {
            sel = k;
            cum_s -= bs[k];  // the carry of the next pass: weights >= the kept bucket's upper edge
            cum_c -= bc[k];
            break;
        }
        if (k == 0) {  // no crossing within rounding: keep the lowest bucket
            cum_s -= bs[0];
            cum_c -= bc[0];
        }
    }
    const unsigned long long new_lo = x.lo + static_cast<unsigned long long>(sel) * step;
    unsigned long long new_hi = new_lo + step;
    if (new_hi > x.hi) new_hi = x.hi;
    x.lo = new_lo;
    x.hi = new_hi;
    x.carry_sum = cum_s;
    x.carry_cnt = cum_c;
    if (bc[sel] == 0 || step == 1) {
        // no weight strictly inside (lo, hi): excess(t) = A - t K on [lo, hi]
        double t = cum_c > 0 ? (cum_s - x.target) / static_cast<double>(cum_c) : 0.0;
        const double tlo = __longlong_as_double(static_cast<long long>(x.lo));
        const double thi = __longlong_as_double(static_cast<long long>(x.hi));
        x.t = fmin(fmax(t, tlo), thi);
        x.done = 1;
    }
    *st = x;
}

__global__ void k_result(State* st, double* result) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    State x = *st;
    if (!x.done) {  // every pass narrowed the range: lo is the root to the last bit
        x.t = __longlong_as_double(static_cast<long long>(x.lo));
        x.done = 1;
        *st = x;
    }
    result[0] = x.t;
    result[1] = x.S;
    result[2] = x.wmax;
    result[3] = static_cast<double>(x.carry_cnt);
    result[4] = static_cast<double>(x.invalid);
}

__device__ __forceinline__ bool keep(double w, double t, uint64_t seed, uint64_t ev) {
    if (!valid(w)) return false;
    uint4 o = rng::philox4x32_10(make_uint4(static_cast<uint32_t>(ev), static_cast<uint32_t>(ev >> 32), kStream, 0u),
                                 static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
    return rng::unit_from_bits(o.y, o.x) * t < w;
}

__global__ void __launch_bounds__(kThreads) k_count(const double* w, int64_t n, const double* tmax, uint64_t seed,
                                                    uint64_t ev0, long long* counts) {
    __shared__ int sc[kThreads];
    const double t = *tmax;
    const int64_t e0 = blockIdx.x * static_cast<int64_t>(kSelBlock) + threadIdx.x * kSelPerThread;
    int c = 0;
    for (int k = 0; k < kSelPerThread; ++k) {
        const int64_t e = e0 + k;
        if (e < n && keep(w[e], t, seed, ev0 + static_cast<uint64_t>(e))) ++c;
    }
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sc[threadIdx.x] += sc[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[blockIdx.x] = sc[0];
}

// exclusive scan of the block counts (one block), total into n_out
__global__ void __launch_bounds__(1024) k_scan(const long long* counts, int64_t nb, long long* offsets,
                                               int64_t* n_out) {
    __shared__ long long s[1024];
    const int64_t per = (nb + 1023) / 1024;
    const int64_t a = threadIdx.x * per, b = min(nb, a + per);
    long long loc = 0;
    for (int64_t i = a; i < b; ++i) loc += counts[i];
    s[threadIdx.x] = loc;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        long long v = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    long long run = s[threadIdx.x] - loc;  // exclusive prefix of this thread's segment
    for (int64_t i = a; i < b; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
    if (threadIdx.x == 1023) *n_out = s[1023];
}

__global__ void __launch_bounds__(kThreads) k_write(const double* w, int64_t n, const double* tmax, uint64_t seed,
                                                    uint64_t ev0, const long long* offsets, int64_t* idx,
                                                    double* wout) {
    __shared__ int sc[kThreads];
    const double t = *tmax;
    const int64_t e0 = blockIdx.x * static_cast<int64_t>(kSelBlock) + threadIdx.x * kSelPerThread;
    unsigned mask = 0;
    for (int k = 0; k < kSelPerThread; ++k) {
        const int64_t e = e0 + k;
        if (e < n && keep(w[e], t, seed, ev0 + static_cast<uint64_t>(e))) mask |= 1u << k;
    }
    const int c = __popc(mask);
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < kThreads; o <<= 1) {
        int v = threadIdx.x >= o ? sc[threadIdx.x - o] : 0;
        __syncthreads();
        sc[threadIdx.x] += v;
        __syncthreads();
    }
    long long pos = offsets[blockIdx.x] + sc[threadIdx.x] - c;
    for (int k = 0; k < kSelPerThread; ++k) {
        if (mask & (1u << k)) {
            const int64_t e = e0 + k;
            idx[pos] = e;
            wout[pos] = fmax(w[e], t);
            ++pos;
        }
    }
}

}  // namespace uw
}  // namespace ps

using namespace ps::uw;

namespace {
thread_local std::string u_err;
int ufail(int code, const std::string& m) {
    u_err = m;
    return code;
}
int ucheck(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return PS_OK;
    return ufail(PS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
constexpr size_t kStateBytes = 256;
constexpr size_t kPartBytes = sizeof(double) * 3 * kGrid;
constexpr size_t kHistBytes = (sizeof(double) + sizeof(unsigned int)) * kGrid * kBuckets;
size_t align256(size_t x) { return (x + 255) / 256 * 256; }
int64_t sel_blocks(int64_t n) { return (n + kSelBlock - 1) / kSelBlock; }
}  // namespace

extern "C" {

const char* ps_unweight_last_error(void) { return u_err.c_str(); }

int ps_unweight_workspace_size(int64_t n, size_t* bytes) {
    if (n < 0 || !bytes) return ufail(PS_ERR_INVALID_ARGUMENT, "ps_unweight_workspace_size: bad arguments");
    const size_t sel = align256(sizeof(long long) * static_cast<size_t>(std::max<int64_t>(1, sel_blocks(n)))) * 2;
    *bytes = kStateBytes + align256(kPartBytes) + align256(kHistBytes) + sel;
    return PS_OK;
}

int ps_unweight_max(const double* w, int64_t n, double eps, double* result, void* workspace, size_t ws_bytes,
                    void* stream) {
    size_t need = 0;
    if (!result || n < 0 || (n > 0 && !w) || !(eps >= 0.0) || !workspace ||
        ps_unweight_workspace_size(n, &need) != PS_OK || ws_bytes < need ||
        (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return ufail(PS_ERR_INVALID_ARGUMENT, "ps_unweight_max: bad arguments or workspace");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(workspace);
    State* state = reinterpret_cast<State*>(base);
    double* part = reinterpret_cast<double*>(base + kStateBytes);
    double* hsum = reinterpret_cast<double*>(base + kStateBytes + align256(kPartBytes));
    unsigned int* hcnt = reinterpret_cast<unsigned int*>(hsum + static_cast<size_t>(kGrid) * kBuckets);
    k_partials<<<kGrid, kThreads, 0, st>>>(w, n, part);
    k_init<<<1, 32, 0, st>>>(part, eps, state);
    for (int p = 0; p < kPasses; ++p) {
        k_hist<<<kGrid, kThreads, 0, st>>>(w, n, state, hsum, hcnt);
        k_decide<<<1, kBuckets, 0, st>>>(hsum, hcnt, state);
    }
    k_result<<<1, 32, 0, st>>>(state, result);
    ps::count_launches(3 + 2 * kPasses);
    return ucheck(cudaGetLastError(), "ps_unweight_max");
}

int ps_unweight_select(const double* w, int64_t n, const double* w_max, uint64_t seed, uint64_t event_offset,
                       int64_t* idx, double* w_out, int64_t* n_accepted, void* workspace, size_t ws_bytes,
                       void* stream) {
    size_t need = 0;
    if (n < 0 || (n > 0 && (!w || !idx || !w_out)) || !w_max || !n_accepted || !workspace ||
        ps_unweight_workspace_size(n, &need) != PS_OK || ws_bytes < need ||
        (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return ufail(PS_ERR_INVALID_ARGUMENT, "ps_unweight_select: bad arguments or workspace");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nb = sel_blocks(n);
    if (nb == 0) return ucheck(cudaMemsetAsync(n_accepted, 0, sizeof(int64_t), st), "ps_unweight_select");
    char* base = static_cast<char*>(workspace) + kStateBytes + align256(kPartBytes) + align256(kHistBytes);
    long long* counts = reinterpret_cast<long long*>(base);
    long long* offsets = reinterpret_cast<long long*>(base + align256(sizeof(long long) * nb));
    k_count<<<static_cast<unsigned>(nb), kThreads, 0, st>>>(w, n, w_max, seed, event_offset, counts);
    k_scan<<<1, 1024, 0, st>>>(counts, nb, offsets, n_accepted);
    k_write<<<static_cast<unsigned>(nb), kThreads, 0, st>>>(w, n, w_max, seed, event_offset, offsets, idx, w_out);
    ps::count_launches(3);
    return ucheck(cudaGetLastError(), "ps_unweight_select");
}

}  // extern "C"
