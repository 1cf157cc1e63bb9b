// unweight.cu -- event unweighting on the GPU (Sec. "Unweighting and file output").
//
// Maximum weight with a bounded over-weight share: w_max(eps) is the smallest t >= 0 with
//     sum_b max(0, w_b - t) <= eps * sum_b w_b.
// The excess is continuous and decreasing in t.  Non-negative doubles order like their bit
// patterns, so the root is located by a radix search over the bits of t, most significant byte
// first: pass p splits the current range [lo, lo + 2^(64-8p)) into 256 buckets by the byte at
// bits 56-8p, histograms count and sum of the weights per bucket, and keeps the bucket in which
// the excess crosses eps S (the excess at a bucket's lower edge T follows from the counts and sums
// of all weights >= T).  The search stops when the kept bucket holds no weight (or is one bit
// pattern wide); then no weight lies strictly between the root and the bucket's upper edge, and
// w_max = (A - eps S) / K in closed form, A and K the sum and count of the weights above.  At most
// 8 passes.
//
// The bucket sums are exact integers: a weight m 2^(e-1075) (53-bit significand m, exponent
// field e) enters its bucket as m 2^(e-E) in units of 2^(E-1075), E the exponent field of the
// bucket's largest bit pattern, accumulated in 128 bits.  Integer addition does not depend on
// order, so the result is reproducible bit for bit; the truncation of the
// low bits of weights below the bucket's top binade costs at most one unit of 2^(E-1075) per
// weight (relative 2^-48 of a bucket sum spanning up to 16 binades).  The total sum and the
// maximum are per-block partials over a fixed grid, combined in block order.
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
constexpr int kBuckets = 256;
constexpr int kPasses = 8;
constexpr int kSelPerThread = 8;    // events per thread in the select kernels
constexpr int kSelBlock = kThreads * kSelPerThread;
constexpr uint32_t kStream = 0x556E7700u;

struct State {
    unsigned long long lo, hi;          // current bit range of the root, [lo, hi)
    int shift;                          // the bucket digit of the next pass: bits shift .. shift+7
    double S, target, wmax;
    double carry_sum;                   // sum and count of the weights >= hi
    unsigned long long carry_cnt;
    unsigned long long invalid;
    double t;                           // the result once done
    int done;
};

// finite and non-negative, decided on the bit pattern (sign clear, exponent field not all ones)
__device__ __forceinline__ bool valid_bits(unsigned long long u) { return (u >> 52) < 0x7FFULL; }
__device__ __forceinline__ bool valid(double w) {
    return valid_bits(static_cast<unsigned long long>(__double_as_longlong(w)));
}

// exponent field of the largest bit pattern of bucket j (the bucket's fixed-point unit)
__device__ __forceinline__ int bucket_exp(unsigned long long lo, unsigned long long step, unsigned long long hi, int j) {
    unsigned long long top = lo + static_cast<unsigned long long>(j + 1) * step;  // wraps to 0 only at 2^64
    if (top == 0 || top > hi) top = hi;
    return static_cast<int>((top - 1) >> 52);
}

// significand of a non-negative finite double scaled to units of 2^(E-1075)
// (subnormals have the unit of exponent field 1; a bucket of subnormals only uses that unit)
__device__ __forceinline__ unsigned long long fixed_units(unsigned long long u, int E) {
    const int e = static_cast<int>(u >> 52);
    const unsigned long long m = (u & 0xFFFFFFFFFFFFFULL) | (e > 0 ? (1ULL << 52) : 0ULL);
    const int sh = (E > 0 ? E : 1) - (e > 0 ? e : 1);
    return sh >= 64 ? 0ULL : (m >> sh);
}

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

// combine the block partials: a fixed-order tree over kGrid entries (kGrid threads)
__global__ void __launch_bounds__(kGrid) k_init(const double* part, double eps, State* st) {
    __shared__ double ss[kGrid], sm[kGrid], sb[kGrid];
    const int t = threadIdx.x;
    ss[t] = part[3 * t];
    sm[t] = part[3 * t + 1];
    sb[t] = part[3 * t + 2];
    __syncthreads();
    for (int o = kGrid / 2; o > 0; o >>= 1) {
        if (t < o) {
            ss[t] += ss[t + o];
            sm[t] = fmax(sm[t], sm[t + o]);
            sb[t] += sb[t + o];
        }
        __syncthreads();
    }
    if (t != 0) return;
    const double S = ss[0], m = sm[0], bad = sb[0];
    State s{};
    s.S = S;
    s.wmax = m;
    s.invalid = static_cast<unsigned long long>(bad);
    s.target = eps * S;
    s.lo = 0;
    s.hi = static_cast<unsigned long long>(__double_as_longlong(m)) + 1;
    s.shift = 56;
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

// one radix pass: per-block histogram of count and exact sum over the 256 buckets of [lo, hi)
__global__ void __launch_bounds__(kThreads) k_hist(const double* w, int64_t n, const State* st,
                                                   unsigned long long* hlo, unsigned long long* hhi,
                                                   unsigned int* hcnt) {
    // warp-private histograms: no contention between warps on a crowded bucket
    __shared__ unsigned long long slo[kThreads / 32][kBuckets], shi[kThreads / 32][kBuckets];
    __shared__ unsigned int sc[kThreads / 32][kBuckets];
    __shared__ int sexp[kBuckets];
    if (st->done) return;
    const unsigned long long lo = st->lo, hi = st->hi;
    const int shift = st->shift;
    const unsigned long long step = 1ULL << shift;
    for (int j = threadIdx.x; j < kBuckets; j += kThreads) sexp[j] = bucket_exp(lo, step, hi, j);
    for (int j = threadIdx.x; j < (kThreads / 32) * kBuckets; j += kThreads) {
        slo[j / kBuckets][j % kBuckets] = 0;
        shi[j / kBuckets][j % kBuckets] = 0;
        sc[j / kBuckets][j % kBuckets] = 0;
    }
    __syncthreads();
    const int64_t chunk = (n + kGrid - 1) / kGrid;
    const int64_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = b0; base < b1; base += kThreads) {  // block-uniform trip count (warp collectives)
        const int64_t i = base + threadIdx.x;
        const unsigned long long u = i < b1 ? static_cast<unsigned long long>(__double_as_longlong(w[i])) : ~0ULL;
        const bool in = valid_bits(u) && u >= lo && u < hi;
        const int bk = in ? static_cast<int>((u - lo) >> shift) : -1;
        const unsigned long long v = in ? fixed_units(u, sexp[bk]) : 0ULL;
        // lanes of one bucket combine first: exact 21-bit limb sums, one leader per bucket
        const unsigned grp = __match_any_sync(0xffffffffu, bk);
        const unsigned l0 = __reduce_add_sync(grp, static_cast<unsigned>(v & 0x1FFFFF));
        const unsigned l1 = __reduce_add_sync(grp, static_cast<unsigned>((v >> 21) & 0x1FFFFF));
        const unsigned l2 = __reduce_add_sync(grp, static_cast<unsigned>(v >> 42));
        if (in && lane == __ffs(grp) - 1) {
            // sum = l0 + l1 2^21 + l2 2^42 < 2^64 * 2^5: low 64 bits and the carry out
            const unsigned long long t1 = static_cast<unsigned long long>(l1) << 21;
            const unsigned long long t2 = static_cast<unsigned long long>(l2) << 42;
            unsigned long long sum = static_cast<unsigned long long>(l0) + t1;
            unsigned long long carry = 0;
            const unsigned long long s2 = sum + t2;
            if (s2 < sum) ++carry;
            carry += static_cast<unsigned long long>(l2) >> 22;  // bits of l2 2^42 above 2^64
            sum = s2;
            // one leader per bucket in this warp and the histogram private to the warp: plain
            // read-modify-write, no atomics
            const unsigned long long old = slo[warp][bk];
            slo[warp][bk] = old + sum;
            if (old + sum < old) ++carry;
            shi[warp][bk] += carry;
            sc[warp][bk] += static_cast<unsigned>(__popc(grp));
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kBuckets; j += kThreads) {
        unsigned long long l = 0, h = 0;
        unsigned int c = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            const unsigned long long v = slo[w][j];
            l += v;
            if (l < v) ++h;
            h += shi[w][j];
            c += sc[w][j];
        }
        hlo[blockIdx.x * kBuckets + j] = l;
        hhi[blockIdx.x * kBuckets + j] = h;
        hcnt[blockIdx.x * kBuckets + j] = c;
    }
}

// combine the block histograms (exact 128-bit sums) and choose the bucket holding the root
constexpr int kDecideSplit = 4;  // threads per bucket when combining the block histograms

__global__ void __launch_bounds__(kBuckets * kDecideSplit) k_decide(const unsigned long long* hlo,
                                                                   const unsigned long long* hhi,
                                                                   const unsigned int* hcnt, State* st) {
    __shared__ double bs[kBuckets];
    __shared__ unsigned long long bc[kBuckets];
    __shared__ unsigned long long plo[kDecideSplit][kBuckets], phi[kDecideSplit][kBuckets], pc[kDecideSplit][kBuckets];
    if (st->done) return;
    const int j = threadIdx.x % kBuckets, part = threadIdx.x / kBuckets;
    const unsigned long long step0 = 1ULL << st->shift;
    {
        unsigned long long l = 0, h = 0, c = 0;
        for (int b = part; b < kGrid; b += kDecideSplit) {
            const unsigned long long v = hlo[b * kBuckets + j];
            l += v;
            if (l < v) ++h;
            h += hhi[b * kBuckets + j];
            c += hcnt[b * kBuckets + j];
        }
        plo[part][j] = l;
        phi[part][j] = h;
        pc[part][j] = c;
    }
    __syncthreads();
    if (part != 0) return;
    unsigned long long slo = 0, shi = 0, c = 0;
    for (int k = 0; k < kDecideSplit; ++k) {
        const unsigned long long v = plo[k][j];
        slo += v;
        if (slo < v) ++shi;
        shi += phi[k][j];
        c += pc[k][j];
    }
    // value = (shi 2^64 + slo) 2^(E - 1075)
    const int E = bucket_exp(st->lo, step0, st->hi, j);
    const int scale = (E > 0 ? E : 1) - 1075;
    bs[j] = ldexp(static_cast<double>(shi) * 18446744073709551616.0 + static_cast<double>(slo), scale);
    bc[j] = c;
    asm volatile("bar.sync 1, %0;\n" ::"r"(kBuckets));  // the kBuckets threads of part 0
    if (j != 0) return;
    State x = *st;
    const unsigned long long step = 1ULL << x.shift;
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
    x.shift -= 8;
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
constexpr size_t kHistBytes = (2 * sizeof(unsigned long long) + sizeof(unsigned int)) * kGrid * kBuckets;
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
    unsigned long long* hlo = reinterpret_cast<unsigned long long*>(base + kStateBytes + align256(kPartBytes));
    unsigned long long* hhi = hlo + static_cast<size_t>(kGrid) * kBuckets;
    unsigned int* hcnt = reinterpret_cast<unsigned int*>(hhi + static_cast<size_t>(kGrid) * kBuckets);
    k_partials<<<kGrid, kThreads, 0, st>>>(w, n, part);
    k_init<<<1, kGrid, 0, st>>>(part, eps, state);
    for (int p = 0; p < kPasses; ++p) {
        k_hist<<<kGrid, kThreads, 0, st>>>(w, n, state, hlo, hhi, hcnt);
        k_decide<<<1, kBuckets * kDecideSplit, 0, st>>>(hlo, hhi, hcnt, state);
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
