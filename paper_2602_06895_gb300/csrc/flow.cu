// flow.cu -- rational-quadratic-spline coupling flow on the GPU: the learned proposal that
// replaces or refines the VEGAS grid (neural importance sampling with rational-quadratic spline
// transformations, Sec. 3.2.2; the spline of Durkan et al. 2019, whose single-bin case is the
// RQF of Sec. 2.3).
//
// Layer l transforms the dims B_l with a monotone spline on [0,1] whose K widths, K heights and
// K+1 knot derivatives come from an MLP of the other dims A_l:
//     A -> Linear(H) -> SiLU -> Linear(H) -> SiLU -> Linear(|B| (3K+1)).
// The MLP GEMMs run on the tensor cores in bfloat16 with FP32 accumulation (warp-level
// mma.sync m16n8k16, with bias, SiLU and the bfloat16 copy of the activation fused into the
// epilogue); the spline, its log-determinant and the backward pass run in FP32.
//
// Training minimises the importance-weighted forward KL  L = sum_b c_b sum_l sum_{j in B_l}
// log F_l'(x_j^(l)),  c_b = w_b / sum w,  w_b = f J_map / g  on samples the flow itself drew
// (r fixed).  The inverse chain r -> z is the stored forward chain; the backward sweep runs
// l = 0 .. L-1 with the implicit-function rule  d x^(l) / d x^(l+1) = 1/F',  d x^(l)/d theta =
// -F_theta/F',  and the derivatives F_theta, F'_theta, F'' of the bin formula are obtained by
// forward-mode differentiation (dual numbers with 7 tangents) of the spline formula itself.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "philox.cuh"
#include "ps.h"

namespace ps {
void count_launches(int n);
namespace flow {

constexpr int kMaxDims = 24;
constexpr int kMaxLayers = 8;
constexpr int kMaxBins = 32;
constexpr float kMinW = 1e-3f, kMinH = 1e-3f, kMinD = 1e-3f;
constexpr int kInPad = 16;  // MLP input width (conditioning dims, zero padded)

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------------------------------
// BF16 tensor-core GEMM: C[m, n] = sum_k A(m, k) B(n, k) (+ bias[n]), A(m,k) = A[m*lam + k*lak],
// B(n,k) = B[n*lbn + k*lbk]; 64x64 tile per CTA (4 warps of 32x32), K in steps of 32 through
// shared memory; FP32 accumulate; epilogue: fp32 store or atomic add, and a bfloat16 copy of
// the (optionally SiLU-activated) result.  grid.z splits K (for the batch-long weight
// gradients, which accumulate with atomics).
struct GemmArgs {
    const bf16* A;
    int64_t lam, lak;
    const bf16* B;
    int64_t lbn, lbk;
    int M, N, K;
    int kchunk;
    const float* bias;
    float* C;
    int64_t ldc;
    bf16* Cb;
    int64_t ldcb;
    int act;      // 1: SiLU on the bf16 copy; 2: C and its copy times SiLU'(Zs) (backward)
    const float* Zs;  // pre-activations for act == 2, [M][ldc]
    int atomic;   // 1: atomicAdd into C
    int trans_c;  // 1: C(m, n) stored at C[n * ldc + m] (fp32 only)
    int a_vec, b_vec;  // 1: the operand's base is 16-byte aligned (16-byte loads allowed)
};

// The hardware base-2 exponential and reciprocal (a few ulp in FP32).  Every exponential of the
// flow is taken as 2^(x log2 e), with the same roundings in every kernel, so that the fused
// sampling layers and the layer-by-layer kernels compute identical activations and splines.
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;\n" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;\n" : "=f"(r) : "f"(x));
    return r;
}
constexpr float kLog2e = 1.4426950408889634f;

// SiLU x sigma(x) = x / (1 + 2^(-x log2 e)) (a few ulp in FP32, far below the bfloat16 rounding
// that follows); for x -> -inf the denominator overflows and the result is 0.
__device__ __forceinline__ float silu(float x) { return x * rcp_approx(1.0f + ex2_approx(x * -kLog2e)); }
__device__ __forceinline__ float silu_grad(float x) {
    const float s = rcp_approx(1.0f + ex2_approx(x * -kLog2e));
    return s * (1.0f + x * (1.0f - s));
}

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One operand tile (64 rows x 32 k) moves through registers as 2 x 8 bf16 per thread: eight
// consecutive elements along the operand's unit-stride dimension (k if lk == 1, else rows if
// lr == 1), as one 16-byte load when they are in range and aligned, else element by element
// (zero outside the operand).
struct TileRegs {
    uint4 v[2];
};

__device__ __forceinline__ bool along_k(int64_t lr, int64_t lk) { return lk == 1 || lr != 1; }

__device__ __forceinline__ void fetch_tile(const bf16* X, int64_t lr, int64_t lk, int r0, int R, int k0, int kend,
                                           bool vec, int tid, TileRegs& t) {
    const bool ak = along_k(lr, lk);
    const bf16 zero = __float2bfloat16(0.0f);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int v = tid + i * 128;
        const int r = ak ? v >> 2 : (v & 7) * 8;
        const int k = ak ? (v & 3) * 8 : v >> 3;
        const int gr = r0 + r, gk = k0 + k;
        const int64_t off = static_cast<int64_t>(gr) * lr + static_cast<int64_t>(gk) * lk;
        const bool full = ak ? (lk == 1 && gr < R && gk + 8 <= kend) : (gk < kend && gr + 8 <= R);
        if (vec && full && (off & 7) == 0) {
            t.v[i] = *reinterpret_cast<const uint4*>(X + off);
        } else {
            __align__(16) bf16 e[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int rr = ak ? gr : gr + j, kk = ak ? gk + j : gk;
                e[j] = (rr < R && kk < kend) ? X[static_cast<int64_t>(rr) * lr + static_cast<int64_t>(kk) * lk] : zero;
            }
            t.v[i] = *reinterpret_cast<const uint4*>(e);
        }
    }
}

__device__ __forceinline__ void store_tile(bf16 (*S)[40], int64_t lr, int64_t lk, int tid, const TileRegs& t) {
    const bool ak = along_k(lr, lk);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int v = tid + i * 128;
        if (ak) {
            *reinterpret_cast<uint4*>(&S[v >> 2][(v & 3) * 8]) = t.v[i];
        } else {
            const bf16* e = reinterpret_cast<const bf16*>(&t.v[i]);
            const int r = (v & 7) * 8, k = v >> 3;
#pragma unroll
            for (int j = 0; j < 8; ++j) S[r + j][k] = e[j];
        }
    }
}

__global__ void __launch_bounds__(128) k_gemm(const GemmArgs g) {
    __shared__ __align__(16) bf16 As[64][40];
    __shared__ __align__(16) bf16 Bs[64][40];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gq = lane >> 2, tq = lane & 3;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    const int k_begin = blockIdx.z * g.kchunk;
    const int k_end = min(g.K, k_begin + g.kchunk);
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;
    TileRegs ra, rb;
    if (k_begin < k_end) {
        fetch_tile(g.A, g.lam, g.lak, m0, g.M, k_begin, k_end, g.a_vec, tid, ra);
        fetch_tile(g.B, g.lbn, g.lbk, n0, g.N, k_begin, k_end, g.b_vec, tid, rb);
        store_tile(As, g.lam, g.lak, tid, ra);
        store_tile(Bs, g.lbn, g.lbk, tid, rb);
    }
    __syncthreads();
    for (int k0 = k_begin; k0 < k_end; k0 += 32) {
        const bool more = k0 + 32 < k_end;
        if (more) {  // next tile's global loads overlap this tile's MMAs
            fetch_tile(g.A, g.lam, g.lak, m0, g.M, k0 + 32, k_end, g.a_vec, tid, ra);
            fetch_tile(g.B, g.lbn, g.lbk, n0, g.N, k0 + 32, k_end, g.b_vec, tid, rb);
        }
#pragma unroll
        for (int ks = 0; ks < 32; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                int r = wm + i * 16 + gq;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int n = wn + j * 8 + gq;
                bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][ks + 2 * tq]);
                bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
        if (more) {
            store_tile(As, g.lam, g.lak, tid, ra);
            store_tile(Bs, g.lbn, g.lbk, tid, rb);
        }
        __syncthreads();
    }
    // epilogue: element pairs (row, col..col+1) as one 8-byte / 4-byte store where the row is
    // complete and aligned, else element by element
    const bool pair_ok = !g.atomic && !g.trans_c && (g.ldc % 2 == 0) && (g.ldcb % 2 == 0) &&
                         (reinterpret_cast<uintptr_t>(g.C) & 7) == 0 && (reinterpret_cast<uintptr_t>(g.Cb) & 3) == 0;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm + i * 16 + gq + 8 * h;
                const int col = n0 + wn + j * 8 + 2 * tq;
                if (row >= g.M) continue;
                float v[2] = {acc[i][j][2 * h], acc[i][j][2 * h + 1]};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (g.bias && blockIdx.z == 0 && col + e < g.N) v[e] += g.bias[col + e];
                    if (g.act == 2 && col + e < g.N) v[e] *= silu_grad(g.Zs[row * g.ldc + col + e]);
                }
                if (pair_ok && col + 1 < g.N) {
                    if (g.C) *reinterpret_cast<float2*>(g.C + row * g.ldc + col) = make_float2(v[0], v[1]);
                    if (g.Cb) {
                        const float a0 = g.act == 1 ? silu(v[0]) : v[0], a1 = g.act == 1 ? silu(v[1]) : v[1];
                        *reinterpret_cast<__nv_bfloat162*>(g.Cb + row * g.ldcb + col) = __floats2bfloat162_rn(a0, a1);
                    }
                    continue;
                }
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (col + e >= g.N) continue;
                    if (g.atomic) {
                        atomicAdd(g.C + row * g.ldc + col + e, v[e]);
                    } else if (g.trans_c) {
                        g.C[(col + e) * g.ldc + row] = v[e];
                    } else {
                        if (g.C) g.C[row * g.ldc + col + e] = v[e];
                        if (g.Cb) g.Cb[row * g.ldcb + col + e] = __float2bfloat16(g.act == 1 ? silu(v[e]) : v[e]);
                    }
                }
            }
}

// ------------------------------------------------------------------------------------------
// Backward-pass GEMM: C[m, n] = sum_k A(m, k) B(k, n) with A(m, k) = A[m*lam + k*lak], unit
// stride along k (lak == 1, "AK") or along m (lam == 1, "AM"), and B(k, n) = B[k*ldb + n].
// BF16 operands, FP32 accumulation on mma.sync m16n8k16.  A CTA of 256 threads (8 warps)
// computes a 128 x BN tile.  K moves through shared memory in steps of 32 with a three-stage
// cp.async pipeline of 16-byte copies (zero-filled past the matrix edges), and ldmatrix feeds
// the fragments (transposing where the unit stride is not along k).  Each shared-memory row is
// stored with its 16-byte chunks XOR-permuted by the row index, so that the eight rows of one
// ldmatrix phase fall in eight different bank groups.  Epilogues: atomic add (the split-K
// weight gradients), the SiLU'-scaled BF16 adjoint with the column sums of the bias gradient,
// or a plain FP32 store.  The split-K form with A unit-stride along k can also add the row sums
// of A as its tiles pass through shared memory (the last layer's bias gradient from the
// BF16 adjoint, without a second pass over it).
namespace bwg {
constexpr int kBM = 128, kBK = 32, kStages = 3, kThreads = 256;
enum Epi { kAtomic = 0, kSiluGrad = 1, kStore = 2 };

struct Args {
    const bf16* A;
    int64_t lam, lak;
    const bf16* B;
    int64_t ldb;
    int M, N, K, kchunk;
    float* C;          // kAtomic, kStore
    int64_t ldc;
    const float* Zs;   // kSiluGrad: pre-activations Z[m * ldz + n]
    int64_t ldz;
    bf16* Cb;          // kSiluGrad: the adjoint as bfloat16, Cb[m * ldcb + n]
    int64_t ldcb;
    float* colsum;     // kSiluGrad: column sums of the adjoint (bias gradient), atomic
    float* rowsum;     // kAtomic with A unit-stride along k: row sums of A (bias gradient), atomic
};

constexpr size_t smem_bytes(int bn) { return static_cast<size_t>(kStages) * (kBM * kBK + kBK * bn) * sizeof(bf16); }

__device__ __forceinline__ void cp16(bf16* dst, const bf16* src, int bytes) {
    const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
__device__ __forceinline__ void ldsm4(uint32_t* r, const bf16* p) {
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm4t(uint32_t* r, const bf16* p) {
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// shared-memory element offsets of the 16-byte chunk (row, chunk) in the three tile layouts:
// A as [128 m][32 k] (AK), A as [32 k][128 m] (AM), B as [32 k][BN n]
__device__ __forceinline__ int off_ak(int m, int c) { return m * kBK + ((c ^ ((m >> 1) & 3)) << 3); }
__device__ __forceinline__ int off_am(int k, int c) { return k * kBM + ((c ^ (k & 7)) << 3); }
template <int BN>
__device__ __forceinline__ int off_b(int k, int c) {
    if constexpr (BN == 16) return k * 16 + ((c ^ ((k >> 2) & 1)) << 3);
    else return k * BN + ((c ^ (k & 7)) << 3);
}

// one stage: the A and B tiles of k in [kb, kb + 32) clipped to [.., k_end)
template <int BN, bool kAM>
__device__ __forceinline__ void load_stage(const Args& g, bf16* As, bf16* Bs, int m0, int n0, int kb, int k_end,
                                           int tid) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {  // A: 512 chunks of 8 elements
        const int id = tid + i * kThreads;
        if constexpr (!kAM) {
            const int r = id >> 2, c = id & 3;
            const int m = m0 + r, k = kb + c * 8;
            const int valid = (m < g.M) ? max(0, min(8, k_end - k)) : 0;
            const bf16* src = valid > 0 ? g.A + static_cast<int64_t>(m) * g.lam + k : g.A;
            cp16(As + off_ak(r, c), src, 2 * valid);
        } else {
            const int r = id >> 4, c = id & 15;
            const int k = kb + r, m = m0 + c * 8;
            const int valid = (k < k_end) ? max(0, min(8, g.M - m)) : 0;
            const bf16* src = valid > 0 ? g.A + static_cast<int64_t>(k) * g.lak + m : g.A;
            cp16(As + off_am(r, c), src, 2 * valid);
        }
    }
    constexpr int kBChunks = kBK * BN / 8;  // B: 512 (BN 128) or 64 (BN 16) chunks
#pragma unroll
    for (int i = 0; i < (kBChunks + kThreads - 1) / kThreads; ++i) {
        const int id = tid + i * kThreads;
        if (id < kBChunks) {
            const int r = id / (BN / 8), c = id % (BN / 8);
            const int k = kb + r, n = n0 + c * 8;
            const int valid = (k < k_end) ? max(0, min(8, g.N - n)) : 0;
            const bf16* src = valid > 0 ? g.B + static_cast<int64_t>(k) * g.ldb + n : g.B;
            cp16(Bs + off_b<BN>(r, c), src, 2 * valid);
        }
    }
}

template <int BN, bool kAM, int kEpi>
__global__ void __launch_bounds__(kThreads, 2) k_gemm_bw(const __grid_constant__ Args g, int pairs) {
    constexpr int WN = BN == 16 ? 1 : 4, WM = 8 / WN;  // warp grid
    constexpr int TM = kBM / WM, TN = BN / WN;         // warp tile
    constexpr int MI = TM / 16, NJ = TN / 8;
    static_assert(NJ % 2 == 0, "B fragments come in pairs of n8 tiles");
    extern __shared__ __align__(128) bf16 sm[];
    bf16* As = sm;                            // kStages x [kBM * kBK]
    bf16* Bs = sm + kStages * kBM * kBK;      // kStages x [kBK * BN]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm0 = (warp / WN) * TM, wn0 = (warp % WN) * TN;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int k_begin = blockIdx.z * g.kchunk;
    const int k_end = min(g.K, k_begin + g.kchunk);
    const int nk = k_end > k_begin ? (k_end - k_begin + kBK - 1) / kBK : 0;
    float acc[MI][NJ][4];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < nk) load_stage<BN, kAM>(g, As + s * kBM * kBK, Bs + s * kBK * BN, m0, n0, k_begin + s * kBK, k_end, tid);
        cp_commit();
    }
    const int mat = lane >> 3, r8 = lane & 7;
    float rs = 0.0f;  // row sums of A: row tid / 2, half tid % 2 of the 32 k of a stage
    for (int kt = 0; kt < nk; ++kt) {
        cp_wait<kStages - 2>();  // stage kt has landed (for this thread's copies) ...
        __syncthreads();         // ... for every thread's, and stage kt - 1 is no longer read
        const int nt = kt + kStages - 1;
        if (nt < nk) {
            const int sb = nt % kStages;
            load_stage<BN, kAM>(g, As + sb * kBM * kBK, Bs + sb * kBK * BN, m0, n0, k_begin + nt * kBK, k_end, tid);
        }
        cp_commit();
        const bf16* A_ = As + (kt % kStages) * kBM * kBK;
        const bf16* B_ = Bs + (kt % kStages) * kBK * BN;
#pragma unroll
        for (int ks = 0; ks < kBK; ks += 16) {
            uint32_t af[MI][4], bfr[NJ][2];
#pragma unroll
            for (int i = 0; i < MI; ++i) {
                const int mb = wm0 + i * 16;
                if constexpr (!kAM) {  // blocks (m, k): mat bit 0 -> m + 8, bit 1 -> k + 8
                    ldsm4(af[i], A_ + off_ak(mb + r8 + (mat & 1) * 8, (ks >> 3) + (mat >> 1)));
                } else {               // stored [k][m], transposed on the load
                    ldsm4t(af[i], A_ + off_am(ks + r8 + (mat >> 1) * 8, (mb >> 3) + (mat & 1)));
                }
            }
#pragma unroll
            for (int j = 0; j < NJ; j += 2) {  // blocks (k, n): mat bit 0 -> k + 8, bit 1 -> n + 8
                uint32_t t[4];
                ldsm4t(t, B_ + off_b<BN>(ks + r8 + (mat & 1) * 8, ((wn0 + j * 8) >> 3) + (mat >> 1)));
                bfr[j][0] = t[0];
                bfr[j][1] = t[1];
                bfr[j + 1][0] = t[2];
                bfr[j + 1][1] = t[3];
            }
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) mma16816(acc[i][j], af[i], bfr[j]);
        }
        if constexpr (kEpi == kAtomic && !kAM) {
            if (g.rowsum != nullptr) {
                const int r = tid >> 1, hc = 2 * (tid & 1);
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const uint4 q = *reinterpret_cast<const uint4*>(A_ + off_ak(r, hc + c));
                    const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float2 f2 = __bfloat1622float2(h2[e]);
                        rs += f2.x + f2.y;
                    }
                }
            }
        }
    }
    cp_wait<0>();
    if constexpr (kEpi == kAtomic && !kAM) {
        if (g.rowsum != nullptr) {
            rs += __shfl_xor_sync(0xffffffffu, rs, 1);
            const int r = tid >> 1;
            if ((tid & 1) == 0 && blockIdx.y == 0 && m0 + r < g.M) atomicAdd(g.rowsum + m0 + r, rs);
        }
    }

    const int gq = lane >> 2, tq = lane & 3;
    float cs[NJ][2];
#pragma unroll
    for (int j = 0; j < NJ; ++j) cs[j][0] = cs[j][1] = 0.0f;
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NJ; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm0 + i * 16 + gq + 8 * h;
                const int col = n0 + wn0 + j * 8 + 2 * tq;
                if (row >= g.M || col >= g.N) continue;
                const bool two = col + 1 < g.N;
                float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
                if constexpr (kEpi == kAtomic) {
                    float* p = g.C + static_cast<int64_t>(row) * g.ldc + col;
                    atomicAdd(p, v0);
                    if (two) atomicAdd(p + 1, v1);
                } else if constexpr (kEpi == kStore) {
                    float* p = g.C + static_cast<int64_t>(row) * g.ldc + col;
                    if (two && pairs) {
                        *reinterpret_cast<float2*>(p) = make_float2(v0, v1);
                    } else {
                        p[0] = v0;
                        if (two) p[1] = v1;
                    }
                } else {
                    const float* z = g.Zs + static_cast<int64_t>(row) * g.ldz + col;
                    bf16* q = g.Cb + static_cast<int64_t>(row) * g.ldcb + col;
                    if (two && pairs) {
                        const float2 zz = *reinterpret_cast<const float2*>(z);
                        v0 *= silu_grad(zz.x);
                        v1 *= silu_grad(zz.y);
                        *reinterpret_cast<__nv_bfloat162*>(q) = __floats2bfloat162_rn(v0, v1);
                    } else {
                        v0 *= silu_grad(z[0]);
                        q[0] = __float2bfloat16(v0);
                        if (two) {
                            v1 *= silu_grad(z[1]);
                            q[1] = __float2bfloat16(v1);
                        } else {
                            v1 = 0.0f;
                        }
                    }
                    cs[j][0] += v0;
                    cs[j][1] += v1;
                }
            }
    if constexpr (kEpi == kSiluGrad) {
        if (g.colsum != nullptr) {  // the warp's column sums: over gq (lane bits 2-4), then one atomic
#pragma unroll
            for (int j = 0; j < NJ; ++j)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    float s = cs[j][e];
                    s += __shfl_xor_sync(0xffffffffu, s, 4);
                    s += __shfl_xor_sync(0xffffffffu, s, 8);
                    s += __shfl_xor_sync(0xffffffffu, s, 16);
                    const int col = n0 + wn0 + j * 8 + 2 * tq + e;
                    if (gq == 0 && col < g.N && m0 + wm0 < g.M) atomicAdd(g.colsum + col, s);
                }
        }
    }
}
}  // namespace bwg

// ------------------------------------------------------------------------------------------
// dual numbers with 7 tangents: (x, x_k, w_k, y_k, h_k, d_k, d_{k+1})
struct Dual {
    float v;
    float t[7];
};
__device__ __forceinline__ Dual dconst(float v) {
    Dual r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < 7; ++i) r.t[i] = 0.0f;
    return r;
}
__device__ __forceinline__ Dual dvar(float v, int i) {
    Dual r = dconst(v);
    r.t[i] = 1.0f;
    return r;
}
__device__ __forceinline__ Dual operator+(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < 7; ++i) r.t[i] = a.t[i] + b.t[i];
    return r;
}
__device__ __forceinline__ Dual operator-(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < 7; ++i) r.t[i] = a.t[i] - b.t[i];
    return r;
}
__device__ __forceinline__ Dual operator*(const Dual& a, const Dual& b) {
    Dual r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < 7; ++i) r.t[i] = a.t[i] * b.v + a.v * b.t[i];
    return r;
}
__device__ __forceinline__ Dual operator/(const Dual& a, const Dual& b) {
    Dual r;
    float ib = 1.0f / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < 7; ++i) r.t[i] = (a.t[i] - r.v * b.t[i]) * ib;
    return r;
}
__device__ __forceinline__ Dual operator*(float s, const Dual& a) {
    Dual r;
    r.v = s * a.v;
#pragma unroll
    for (int i = 0; i < 7; ++i) r.t[i] = s * a.t[i];
    return r;
}

__device__ __forceinline__ Dual operator-(const Dual& a, float b) {
    Dual r = a;
    r.v -= b;
    return r;
}
__device__ __forceinline__ Dual operator*(const Dual& a, float b) { return b * a; }

// The bin formula: y = y_k + h [s xi^2 + d0 xi(1-xi)] / [s + (d1 + d0 - 2s) xi (1-xi)] and its
// derivative F' = s^2 [d1 xi^2 + 2 s xi (1-xi) + d0 (1-xi)^2] / [..]^2, s = h/w, xi = (x-x_k)/w.
// reciprocals of the bin formula: the hardware reciprocal in FP32 (w >= 1e-3, den > 0), exact
// division for the dual numbers of the backward pass
__device__ __forceinline__ float brcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ Dual brcp(const Dual& a) { return dconst(1.0f) / a; }

template <typename T>
__device__ __forceinline__ void bin_eval(const T& x, const T& x0, const T& w, const T& y0, const T& h, const T& d0,
                                         const T& d1, T& F, T& Fp) {
    const T iw = brcp(w);
    T xi = (x - x0) * iw;
    T s = h * iw;
    T om = xi - xi * xi;
    T xm = xi - 1.0f;
    T den = s + (d1 + d0 - 2.0f * s) * om;
    const T iden = brcp(den);
    F = y0 + h * (s * xi * xi + d0 * om) * iden;
    Fp = s * s * (d1 * xi * xi + 2.0f * s * om + d0 * (xm * xm)) * (iden * iden);
}

// softplus and sigmoid with the hardware exponential and logarithm; for a << 0 softplus(a) ~ e^a
// falls below the 1e-3 floor added to the knot derivatives, so log(1 + e^a) rounding to 0 there
// is harmless
__device__ __forceinline__ float softplus(float a) { return a > 20.0f ? a : __logf(1.0f + __expf(a)); }
__device__ __forceinline__ float sigmoid(float a) { return __fdividef(1.0f, 1.0f + __expf(-a)); }

// Raw MLP outputs of one transformed dim are read as raw[i * ld] (parameter-major layout: the
// events of a warp read one parameter row, coalesced): widths 0..K-1, heights K..2K-1, knot
// derivatives 2K..3K.
// e^(a - m) of a softmax, as 2^(a log2 e - m log2 e)
__device__ __forceinline__ float softmax_exp(float a, float nm) { return ex2_approx(fmaf(a, kLog2e, nm)); }

__device__ __forceinline__ void softmax_norm(const float* raw, int64_t ld, int K, float& m, float& iz) {
    m = -INFINITY;
    for (int i = 0; i < K; ++i) m = fmaxf(m, raw[i * ld]);
    const float nm = -m * kLog2e;
    float z = 0.0f;
    for (int i = 0; i < K; ++i) z += softmax_exp(raw[i * ld], nm);
    iz = rcp_approx(z);
}

// The bin holding v among the width knots (v = x) or the height knots (v = y, inverse), with
// its parameters and the softmax quantities the backward pass needs.
struct Bin {
    int k;
    float x0, w, y0, h, d0, d1;
    float mw, iw, mh, ih;  // softmax maxima and inverse sums
    float pw, ph;          // softmax probabilities of bin k
    float sx, sy;          // sums of the softmax probabilities of the bins before k
    float sg0, sg1;        // softplus' (= sigmoid) at the derivative pre-activations of k, k+1
};

__device__ __forceinline__ Bin locate(const float* raw, int64_t ld, int K, float v, bool by_height) {
    Bin b;
    softmax_norm(raw, ld, K, b.mw, b.iw);
    softmax_norm(raw + K * ld, ld, K, b.mh, b.ih);
    const float cw = 1.0f - K * kMinW, chh = 1.0f - K * kMinH;
    float x0 = 0.0f, y0 = 0.0f, sx = 0.0f, sy = 0.0f;
    int k = 0;
    const float nmw = -b.mw * kLog2e, nmh = -b.mh * kLog2e;
    for (;; ++k) {
        float pw = softmax_exp(raw[k * ld], nmw) * b.iw;
        float ph = softmax_exp(raw[(K + k) * ld], nmh) * b.ih;
        float w = kMinW + cw * pw, h = kMinH + chh * ph;
        if (k == K - 1 || (by_height ? v < y0 + h : v < x0 + w)) {
            b.w = w;
            b.h = h;
            b.pw = pw;
            b.ph = ph;
            break;
        }
        x0 += w;
        y0 += h;
        sx += pw;
        sy += ph;
    }
    b.k = k;
    b.x0 = x0;
    b.y0 = y0;
    b.sx = sx;
    b.sy = sy;
    float a0 = raw[(2 * K + k) * ld], a1 = raw[(2 * K + k + 1) * ld];
    b.d0 = kMinD + softplus(a0);
    b.d1 = kMinD + softplus(a1);
    b.sg0 = sigmoid(a0);
    b.sg1 = sigmoid(a1);
    return b;
}

// locate() for a compile-time bin count and unit stride: the raw parameters are read once into
// registers, each exponential is taken once and the bin search is unrolled into selects.  Same
// operations in the same order as locate(), so the results agree bit for bit.
template <int K>
__device__ __forceinline__ Bin locate_fixed(const float* raw, int64_t ld, float v, bool by_height) {
    float w[K], h[K];
    float mw = -INFINITY, mh = -INFINITY;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        w[i] = raw[i * ld];
        h[i] = raw[(K + i) * ld];
        mw = fmaxf(mw, w[i]);
        mh = fmaxf(mh, h[i]);
    }
    float zw = 0.0f, zh = 0.0f;
    const float nmw = -mw * kLog2e, nmh = -mh * kLog2e;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        w[i] = softmax_exp(w[i], nmw);
        h[i] = softmax_exp(h[i], nmh);
    }
#pragma unroll
    for (int i = 0; i < K; ++i) zw += w[i];
#pragma unroll
    for (int i = 0; i < K; ++i) zh += h[i];
    Bin b;
    b.mw = mw;
    b.mh = mh;
    b.iw = rcp_approx(zw);
    b.ih = rcp_approx(zh);
    const float cw = 1.0f - K * kMinW, chh = 1.0f - K * kMinH;
    float cx = 0.0f, cy = 0.0f, csx = 0.0f, csy = 0.0f;
    // branch-free selection of the first bin whose right edge lies above v (the last otherwise):
    // the edges rise strictly, so hit_i = s_i - s_(i-1) with s_i = [v < edge_i] is 1 for that bin
    // alone, and sums of hit_i x value (exact: multiplies by 0 or 1, adds of +0) gather its values
    float g[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float prev = 0.0f;
    int below = 0;  // bins entirely below v: the index of the bin
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const float pw = w[i] * b.iw, ph = h[i] * b.ih;
        const float ww = kMinW + cw * pw, hh = kMinH + chh * ph;
        const float s = (i == K - 1 || (by_height ? v < cy + hh : v < cx + ww)) ? 1.0f : 0.0f;
        const float hit = s - prev;
        below += s == 0.0f ? 1 : 0;
        g[0] = __fmaf_rn(hit, cx, g[0]);
        g[1] = __fmaf_rn(hit, cy, g[1]);
        g[2] = __fmaf_rn(hit, csx, g[2]);
        g[3] = __fmaf_rn(hit, csy, g[3]);
        g[4] = __fmaf_rn(hit, ww, g[4]);
        g[5] = __fmaf_rn(hit, hh, g[5]);
        g[6] = __fmaf_rn(hit, pw, g[6]);
        g[7] = __fmaf_rn(hit, ph, g[7]);
        prev = s;
        cx += ww;
        cy += hh;
        csx += pw;
        csy += ph;
    }
    b.k = below;
    b.x0 = g[0];
    b.y0 = g[1];
    b.sx = g[2];
    b.sy = g[3];
    b.w = g[4];
    b.h = g[5];
    b.pw = g[6];
    b.ph = g[7];
    const float a0 = raw[(2 * K + b.k) * ld], a1 = raw[(2 * K + b.k + 1) * ld];
    b.d0 = kMinD + softplus(a0);
    b.d1 = kMinD + softplus(a1);
    b.sg0 = sigmoid(a0);
    b.sg1 = sigmoid(a1);
    return b;
}

// locate() with the compile-time path when the bin count matches kK
template <int kK>
__device__ __forceinline__ Bin locate_k(const float* raw, int64_t ld, int K, float v, bool by_height) {
    if constexpr (kK > 0) return locate_fixed<kK>(raw, ld, v, by_height);
    else return locate(raw, ld, K, v, by_height);
}

// ------------------------------------------------------------------------------------------
struct LayerDesc {
    int nb, na;             // transformed / conditioning dims
    int tb[kMaxDims];       // transformed dim indices
    int ta[kMaxDims];       // conditioning dim indices
    int P, Ppad;            // raw params per event (nb (3K+1)) and padded row length
    int64_t off_W1, off_b1, off_W2, off_b2, off_W3, off_b3;  // parameter offsets (floats)
};

struct FlowDesc {
    int d, L, K, H;
    LayerDesc layer[kMaxLayers];
};

// z from Philox: dims 2c, 2c+1 from counter (ev_lo, ev_hi, 0x466C6F77 ("Flow"), c), key (seed);
// the top 23 bits k of a word give (k + 1/2) 2^-23 in (0, 1), exact in FP32.
__global__ void k_init_z(int64_t B, int d, uint64_t seed, uint64_t ev0, float* X) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b >= B) return;
    uint64_t ev = ev0 + static_cast<uint64_t>(b);
    for (int j = 0; j < d; j += 2) {
        uint4 o = rng::philox4x32_10(make_uint4(static_cast<uint32_t>(ev), static_cast<uint32_t>(ev >> 32), 0x466C6F77u,
                                                static_cast<uint32_t>(j >> 1)),
                                     static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
        X[b * d + j] = (static_cast<float>(o.x >> 9) + 0.5f) * 0x1p-23f;
        if (j + 1 < d) X[b * d + j + 1] = (static_cast<float>(o.y >> 9) + 0.5f) * 0x1p-23f;
    }
}

__global__ void k_gather(int64_t B, int d, const float* X, const __grid_constant__ LayerDesc ld, bf16* In) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b >= B) return;
    for (int i = 0; i < kInPad; ++i)
        In[b * kInPad + i] = __float2bfloat16(i < ld.na ? X[b * d + ld.ta[i]] : 0.0f);
}

// forward spline of one layer: Xout = Xin with the B dims through F; logdet += sum log F'.
// Praw is parameter-major: raw parameter p of event b at Praw[p * ldp + b].
template <int kK>
__global__ void k_spline_forward(int64_t B, int d, int K, const float* Xin, float* Xout, const float* Praw,
                                 int64_t ldp, const __grid_constant__ LayerDesc ld, float* logdet) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b >= B) return;
    for (int j = 0; j < d; ++j) Xout[b * d + j] = Xin[b * d + j];
    float acc = 0.0f;
    for (int q = 0; q < ld.nb; ++q) {
        const float* raw = Praw + static_cast<int64_t>(q) * (3 * K + 1) * ldp + b;
        int j = ld.tb[q];
        float x = fminf(fmaxf(Xin[b * d + j], 0.0f), 1.0f);
        Bin bn = locate_k<kK>(raw, ldp, K, x, false);
        float F, Fp;
        bin_eval<float>(x, bn.x0, bn.w, bn.y0, bn.h, bn.d0, bn.d1, F, Fp);
        Xout[b * d + j] = fminf(fmaxf(F, 1e-7f), 1.0f - 1e-7f);
        acc += __logf(Fp);
    }
    logdet[b] += acc;
}

// inverse spline of one layer: Xout = Xin with the B dims through F^-1; logq -= sum log F'(x)
template <int kK>
__global__ void k_spline_inverse(int64_t B, int d, int K, const float* Xin, float* Xout, const float* Praw,
                                 int64_t ldp, const __grid_constant__ LayerDesc ld, float* logq) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b >= B) return;
    for (int j = 0; j < d; ++j) Xout[b * d + j] = Xin[b * d + j];
    float acc = 0.0f;
    for (int q = 0; q < ld.nb; ++q) {
        const float* raw = Praw + static_cast<int64_t>(q) * (3 * K + 1) * ldp + b;
        int j = ld.tb[q];
        float y = fminf(fmaxf(Xin[b * d + j], 0.0f), 1.0f);
        Bin bn = locate_k<kK>(raw, ldp, K, y, true);
        // y - y_k = h [s xi^2 + d0 xi (1-xi)] / [s + (d1 + d0 - 2s) xi (1-xi)] is a quadratic in xi;
        // the root in [0,1] in the form free of cancellation: xi = 2c / (-b - sqrt(b^2 - 4ac))
        float s = bn.h / bn.w, dy = y - bn.y0, e = bn.d1 + bn.d0 - 2.0f * s;
        float qa = bn.h * (s - bn.d0) + dy * e, qb = bn.h * bn.d0 - dy * e, qc = -s * dy;
        float disc = fmaxf(qb * qb - 4.0f * qa * qc, 0.0f);
        float den = -qb - sqrtf(disc);
        float xi = den != 0.0f ? fminf(fmaxf(2.0f * qc / den, 0.0f), 1.0f) : 0.0f;
        float x = bn.x0 + xi * bn.w;
        float F, Fp;
        bin_eval<float>(x, bn.x0, bn.w, bn.y0, bn.h, bn.d0, bn.d1, F, Fp);
        Xout[b * d + j] = fminf(fmaxf(x, 0.0f), 1.0f);
        acc += __logf(Fp);
    }
    logq[b] -= acc;
}

// backward of one layer (see the header): inputs x^(l) (Xl), raw params, the adjoint gX of x^(l)
// and the event coefficient c_b = w_b / sum w; outputs the raw-parameter adjoint Gb (bf16, and
// G in fp32 when G is not null; parameter-major like Praw, padding rows zeroed) and the adjoint
// of x^(l+1) in gXn (the conditioning dims get the MLP part later).
template <int kK>
__global__ void k_spline_backward(int64_t B, int d, int K, const float* Xl, const float* Praw, int64_t ldp,
                                  const __grid_constant__ LayerDesc ld, const float* gX, const double* wtot,
                                  const double* wsum, float* G, bf16* Gb, float* gXn, double* loss) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    float lsum = 0.0f;
    if (b < B) {
        const float c = wsum[0] > 0.0 ? static_cast<float>(wtot[b] / wsum[0]) : 0.0f;
        for (int j = 0; j < d; ++j) gXn[b * d + j] = gX[b * d + j];  // A dims pass through
        const float cw = 1.0f - K * kMinW, chh = 1.0f - K * kMinH;
        for (int q = 0; q < ld.nb; ++q) {
            const int64_t row0 = static_cast<int64_t>(q) * (3 * K + 1);
            const float* raw = Praw + row0 * ldp + b;
            int j = ld.tb[q];
            float xv = fminf(fmaxf(Xl[b * d + j], 0.0f), 1.0f);
            Bin bn = locate_k<kK>(raw, ldp, K, xv, false);
            Dual F, Fp;
            bin_eval<Dual>(dvar(xv, 0), dvar(bn.x0, 1), dvar(bn.w, 2), dvar(bn.y0, 3), dvar(bn.h, 4), dvar(bn.d0, 5),
                           dvar(bn.d1, 6), F, Fp);
            float ifp = 1.0f / Fp.v;
            lsum += c * logf(Fp.v);
            float ax = gX[b * d + j] + c * Fp.t[0] * ifp;  // adjoint of x^(l)_j incl. d(c log F')/dx
            gXn[b * d + j] = ax * ifp;                       // d x^(l) / d x^(l+1) = 1/F'
            // bin-parameter adjoints: -a_x F_theta / F' + c F'_theta / F'
            float gt[7];
#pragma unroll
            for (int i = 1; i < 7; ++i) gt[i] = (-ax * F.t[i] + c * Fp.t[i]) * ifp;
            // chain to the raw parameters: x_k = sum_{i<k} w_i and w_k through the width softmax,
            // y_k and h_k through the height softmax, d_k and d_{k+1} through softplus
            const float dotw = gt[1] * bn.sx + gt[2] * bn.pw;
            const float doth = gt[3] * bn.sy + gt[4] * bn.ph;
            float* g = G ? G + row0 * ldp + b : nullptr;
            bf16* gb = Gb + row0 * ldp + b;
            const float nmw = -bn.mw * kLog2e, nmh = -bn.mh * kLog2e;
            for (int i = 0; i < K; ++i) {
                float pw = softmax_exp(raw[i * ldp], nmw) * bn.iw;
                float ph = softmax_exp(raw[(K + i) * ldp], nmh) * bn.ih;
                float aw = i < bn.k ? gt[1] : (i == bn.k ? gt[2] : 0.0f);
                float ah = i < bn.k ? gt[3] : (i == bn.k ? gt[4] : 0.0f);
                float vw = cw * pw * (aw - dotw), vh = chh * ph * (ah - doth);
                if (G) {
                    g[i * ldp] = vw;
                    g[(K + i) * ldp] = vh;
                }
                gb[i * ldp] = __float2bfloat16(vw);
                gb[(K + i) * ldp] = __float2bfloat16(vh);
            }
            for (int i = 0; i <= K; ++i) {
                float v = i == bn.k ? gt[5] * bn.sg0 : (i == bn.k + 1 ? gt[6] * bn.sg1 : 0.0f);
                if (G) g[(2 * K + i) * ldp] = v;
                gb[(2 * K + i) * ldp] = __float2bfloat16(v);
            }
        }
        for (int p = ld.P; p < ld.Ppad; ++p) {
            if (G) G[p * ldp + b] = 0.0f;
            Gb[p * ldp + b] = __float2bfloat16(0.0f);
        }
    }
    // loss = sum_b c_b sum log F'  (one atomic per warp)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, static_cast<double>(lsum));
}

// row sums of an [n][ldm] fp32 matrix over its first B columns into out[n] (atomic; bias
// gradients of the last layer)
__global__ void __launch_bounds__(256) k_rowsum(int64_t B, int64_t ldm, const float* M, float* out) {
    __shared__ float ws[8];
    const int row = blockIdx.y;
    float s = 0.0f;
    for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < B;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x)
        s += M[row * ldm + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < 8; ++w) t += ws[w];
        atomicAdd(out + row, t);
    }
}

// column sums of a [B, n] fp32 matrix into out[n] (atomic; bias gradients)
__global__ void k_colsum(int64_t B, int n, const float* M, float* out) {
    int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= n) return;
    int64_t rows = (B + gridDim.y - 1) / gridDim.y;
    int64_t r0 = blockIdx.y * rows, r1 = min(B, r0 + rows);
    float s = 0.0f;
    for (int64_t r = r0; r < r1; ++r) s += M[r * n + col];
    atomicAdd(out + col, s);
}

__global__ void k_scatter(int64_t B, int d, const __grid_constant__ LayerDesc ld, const float* dIn, float* gXn) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b >= B) return;
    for (int i = 0; i < ld.na; ++i) gXn[b * d + ld.ta[i]] += dIn[b * kInPad + i];
}

// w_b = w_map_b exp(logdet_b) (the flow density is 1/|dr/dz|); block sums into wsum
__global__ void k_weights(int64_t B, const double* wmap, const float* logdet, double* wtot, double* wsum) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    double w = 0.0;
    if (b < B) {
        w = wmap[b] * exp(static_cast<double>(logdet[b]));
        if (!isfinite(w)) w = 0.0;
        wtot[b] = w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(wsum, w);
}

// ------------------------------------------------------------------------------------------
// Fused coupling layer for sampling and density evaluation (no training): one persistent CTA
// per SM holds the layer's weights in shared memory; each warp takes 16 events, runs the three
// GEMMs on the tensor cores with the hidden activations kept in registers (the accumulator
// fragment of two adjacent 8-column tiles is the operand fragment of the next 16-wide k-step),
// stages the raw spline parameters of two transformed dims at a time in shared memory and
// evaluates their splines, and updates X in place (the conditioning dims are never written).
constexpr int kFH = 128;             // hidden width of the fused path
constexpr int kFWarps = 8;
constexpr int kQRows = 56;           // raw rows per transformed dim, padded to 7 tiles of 8
constexpr int kStage = 57;           // staging row stride (floats; odd: conflict-free rows)
constexpr int kW2S = kFH + 8;        // shared row stride (bf16) of W2 and W3
constexpr int kW1S = kInPad + 8;     // shared row stride (bf16) of W1
constexpr int kMaxNb = 8;

struct FusedSmem {
    static constexpr size_t w1 = 0;
    static constexpr size_t w2 = w1 + sizeof(bf16) * kFH * kW1S;
    static constexpr size_t w3 = w2 + sizeof(bf16) * kFH * kW2S;
    static constexpr size_t b1 = w3 + sizeof(bf16) * kMaxNb * kQRows * kW2S;
    static constexpr size_t b2 = b1 + sizeof(float) * kFH;
    static constexpr size_t b3 = b2 + sizeof(float) * kFH;
    static constexpr size_t stage = b3 + sizeof(float) * kMaxNb * kQRows;
    static constexpr size_t total = stage + sizeof(float) * kFWarps * 2 * 16 * kStage;
};

// B-operand fragments of two adjacent 8-column tiles (16 rows n0.., one 16-wide k step at k0) of
// a [n][k] bf16 matrix in shared memory: ldmatrix.x4 of the four 8x8 blocks; r[0..1] belong to
// the tile at n0, r[2..3] to the tile at n0 + 8.
__device__ __forceinline__ void ldsm_b2(uint32_t (&r)[4], const bf16* base, int stride, int n0, int k0, int lane) {
    const int mi = lane >> 3, row = lane & 7;
    const bf16* p = base + (n0 + (mi >> 1) * 8 + row) * stride + k0 + (mi & 1) * 8;
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
// one 8-column tile
__device__ __forceinline__ void ldsm_b1(uint32_t (&r)[2], const bf16* base, int stride, int n0, int k0, int lane) {
    const int mi = (lane >> 3) & 1, row = lane & 7;
    const bf16* p = base + (n0 + row) * stride + k0 + mi * 8;
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

template <bool kInverse, int kK>  // kK: compile-time bin count, or 0 for the runtime K
__global__ void __launch_bounds__(kFWarps * 32, 1)
    k_layer_fused(int64_t B, int d, int K, float* X, float* logdet, const __grid_constant__ LayerDesc ld,
                  const bf16* W1, const float* b1, const bf16* W2, const float* b2, const bf16* W3,
                  const float* b3) {
    extern __shared__ __align__(16) unsigned char smem[];
    bf16* w1s = reinterpret_cast<bf16*>(smem + FusedSmem::w1);
    bf16* w2s = reinterpret_cast<bf16*>(smem + FusedSmem::w2);
    bf16* w3s = reinterpret_cast<bf16*>(smem + FusedSmem::w3);
    float* b1s = reinterpret_cast<float*>(smem + FusedSmem::b1);
    float* b2s = reinterpret_cast<float*>(smem + FusedSmem::b2);
    float* b3s = reinterpret_cast<float*>(smem + FusedSmem::b3);
    float* stage = reinterpret_cast<float*>(smem + FusedSmem::stage);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gq = lane >> 2, tq = lane & 3;
    const int per_q = 3 * K + 1;
    const bf16 zero = __float2bfloat16(0.0f);

    // weights and biases of the layer into shared memory
    for (int i = tid; i < kFH * kInPad; i += blockDim.x) w1s[(i / kInPad) * kW1S + i % kInPad] = W1[i];
    for (int i = tid; i < kFH * kFH / 8; i += blockDim.x) {
        const int r = i / (kFH / 8), c = (i % (kFH / 8)) * 8;
        *reinterpret_cast<uint4*>(w2s + r * kW2S + c) = *reinterpret_cast<const uint4*>(W2 + r * kFH + c);
    }
    for (int i = tid; i < ld.nb * kQRows * (kFH / 8); i += blockDim.x) {
        const int r = i / (kFH / 8), c = (i % (kFH / 8)) * 8;
        const int q = r / kQRows, k = r % kQRows;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (k < per_q) v = *reinterpret_cast<const uint4*>(W3 + (q * per_q + k) * kFH + c);
        *reinterpret_cast<uint4*>(w3s + r * kW2S + c) = v;
    }
    for (int i = tid; i < kFH; i += blockDim.x) {
        b1s[i] = b1[i];
        b2s[i] = b2[i];
    }
    for (int i = tid; i < ld.nb * kQRows; i += blockDim.x) {
        const int q = i / kQRows, k = i % kQRows;
        b3s[i] = k < per_q ? b3[q * per_q + k] : 0.0f;
    }
    __syncthreads();
    (void)zero;

    float* st0 = stage + warp * 2 * 16 * kStage;
    const int64_t n_tiles = (B + 16 * kFWarps - 1) / (16 * kFWarps);
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t e0 = tile * (16 * kFWarps) + warp * 16;
        const int64_t ea = e0 + gq, eb = e0 + gq + 8;
        auto in = [&](int64_t ev, int k) -> float {
            return (ev < B && k < ld.na) ? X[ev * d + ld.ta[k]] : 0.0f;
        };
        uint32_t a0[4];
        a0[0] = pack_bf16(in(ea, 2 * tq), in(ea, 2 * tq + 1));
        a0[1] = pack_bf16(in(eb, 2 * tq), in(eb, 2 * tq + 1));
        a0[2] = pack_bf16(in(ea, 2 * tq + 8), in(ea, 2 * tq + 9));
        a0[3] = pack_bf16(in(eb, 2 * tq + 8), in(eb, 2 * tq + 9));

        // layer 1: 16 x 128, K = 16 (all 16 tiles issued before their epilogues); SiLU; the bf16
        // operand fragments of layer 2
        uint32_t a1[8][4];
        {
            float c[16][4];
#pragma unroll
            for (int p2 = 0; p2 < 8; ++p2) {
                uint32_t bq[4];
                ldsm_b2(bq, w1s, kW1S, 16 * p2, 0, lane);
                const uint32_t b0[2] = {bq[0], bq[1]}, b1v[2] = {bq[2], bq[3]};
#pragma unroll
                for (int e = 0; e < 4; ++e) c[2 * p2][e] = c[2 * p2 + 1][e] = 0.0f;
                mma16816(c[2 * p2], a0, b0);
                mma16816(c[2 * p2 + 1], a0, b1v);
            }
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                const int n = nt * 8;
                const float bb0 = b1s[n + 2 * tq], bb1 = b1s[n + 2 * tq + 1];
                a1[nt >> 1][2 * (nt & 1)] = pack_bf16(silu(c[nt][0] + bb0), silu(c[nt][1] + bb1));
                a1[nt >> 1][2 * (nt & 1) + 1] = pack_bf16(silu(c[nt][2] + bb0), silu(c[nt][3] + bb1));
            }
        }
        // layer 2: 16 x 128, K = 128, eight independent 8-column accumulators per half
        uint32_t a2[8][4];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            float c[8][4];
#pragma unroll
            for (int t = 0; t < 8; ++t) c[t][0] = c[t][1] = c[t][2] = c[t][3] = 0.0f;
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
                for (int p2 = 0; p2 < 4; ++p2) {
                    uint32_t bq[4];
                    ldsm_b2(bq, w2s, kW2S, 64 * half + 16 * p2, 16 * kk, lane);
                    const uint32_t b0[2] = {bq[0], bq[1]}, b1v[2] = {bq[2], bq[3]};
                    mma16816(c[2 * p2], a1[kk], b0);
                    mma16816(c[2 * p2 + 1], a1[kk], b1v);
                }
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int nt = 8 * half + t, n = nt * 8;
                const float bb0 = b2s[n + 2 * tq], bb1 = b2s[n + 2 * tq + 1];
                a2[nt >> 1][2 * (nt & 1)] = pack_bf16(silu(c[t][0] + bb0), silu(c[t][1] + bb1));
                a2[nt >> 1][2 * (nt & 1) + 1] = pack_bf16(silu(c[t][2] + bb0), silu(c[t][3] + bb1));
            }
        }
        // layer 3 and the splines, two transformed dims at a time
        float lsum = 0.0f;
        for (int qp = 0; qp < ld.nb; qp += 2) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int q = qp + s;
                if (q >= ld.nb) break;
                float c[7][4];
#pragma unroll
                for (int t = 0; t < 7; ++t) c[t][0] = c[t][1] = c[t][2] = c[t][3] = 0.0f;
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
#pragma unroll
                    for (int p2 = 0; p2 < 3; ++p2) {
                        uint32_t bq[4];
                        ldsm_b2(bq, w3s, kW2S, q * kQRows + 16 * p2, 16 * kk, lane);
                        const uint32_t b0[2] = {bq[0], bq[1]}, b1v[2] = {bq[2], bq[3]};
                        mma16816(c[2 * p2], a2[kk], b0);
                        mma16816(c[2 * p2 + 1], a2[kk], b1v);
                    }
                    uint32_t bl[2];
                    ldsm_b1(bl, w3s, kW2S, q * kQRows + 48, 16 * kk, lane);
                    mma16816(c[6], a2[kk], bl);
                }
                float* sq = st0 + s * 16 * kStage;
#pragma unroll
                for (int t = 0; t < 7; ++t) {
                    const int col = t * 8 + 2 * tq;
                    const float bb0 = b3s[q * kQRows + col], bb1 = b3s[q * kQRows + col + 1];
                    sq[gq * kStage + col] = c[t][0] + bb0;
                    sq[gq * kStage + col + 1] = c[t][1] + bb1;
                    sq[(gq + 8) * kStage + col] = c[t][2] + bb0;
                    sq[(gq + 8) * kStage + col + 1] = c[t][3] + bb1;
                }
            }
            __syncwarp();
            {
                const int s = lane >> 4, row = lane & 15;
                const int q = qp + s;
                const int64_t ev = e0 + row;
                if (q < ld.nb && ev < B) {
                    const float* raw = st0 + s * 16 * kStage + row * kStage;
                    const int j = ld.tb[q];
                    const float v = fminf(fmaxf(X[ev * d + j], 0.0f), 1.0f);
                    Bin bn = locate_k<kK>(raw, 1, K, v, kInverse);
                    float F, Fp;
                    if (!kInverse) {
                        bin_eval<float>(v, bn.x0, bn.w, bn.y0, bn.h, bn.d0, bn.d1, F, Fp);
                        X[ev * d + j] = fminf(fmaxf(F, 1e-7f), 1.0f - 1e-7f);
                        lsum += __logf(Fp);
                    } else {
                        const float sl = bn.h / bn.w, dy = v - bn.y0, e = bn.d1 + bn.d0 - 2.0f * sl;
                        const float qa = bn.h * (sl - bn.d0) + dy * e, qb = bn.h * bn.d0 - dy * e, qc = -sl * dy;
                        const float disc = fmaxf(qb * qb - 4.0f * qa * qc, 0.0f);
                        const float den = -qb - sqrtf(disc);
                        const float xi = den != 0.0f ? fminf(fmaxf(2.0f * qc / den, 0.0f), 1.0f) : 0.0f;
                        const float x = bn.x0 + xi * bn.w;
                        bin_eval<float>(x, bn.x0, bn.w, bn.y0, bn.h, bn.d0, bn.d1, F, Fp);
                        X[ev * d + j] = fminf(fmaxf(x, 0.0f), 1.0f);
                        lsum -= __logf(Fp);
                    }
                }
            }
            __syncwarp();
        }
        lsum += __shfl_down_sync(0xffffffffu, lsum, 16);
        if (lane < 16 && e0 + lane < B) logdet[e0 + lane] += lsum;
    }
}

// ------------------------------------------------------------------------------------------
// Fused coupling layer on the 5th-generation tensor cores (tcgen05), for sampling and density
// evaluation with hidden width 128 and 16 bins.  A tile is 128 events, one event per TMEM lane:
// the three GEMMs are single-thread tcgen05.mma issues (M = 128; operands in shared memory in the
// K-major canonical layout of 8-row x 16-byte core matrices; FP32 accumulators in TMEM), and each
// epilogue thread reads its own event's row back with tcgen05.ld -- the SiLU of the hidden layers
// writes the next operand tile, and the raw spline parameters of a transformed dim arrive in that
// thread's registers, so the spline needs no staging.
//
// Two tiles are in flight per CTA: the 512 threads form two independent groups of two warpgroups,
// each with its own operand tiles, its own 256 TMEM columns, its own issuing thread, completion
// barriers and named barrier, so that one group's MMAs run on the tensor cores while the other
// group evaluates SiLUs and splines on the CUDA cores.  The weights in shared memory serve both.
// Within a group, warpgroup h takes hidden columns 64h..64h+63 and the transformed dim 2p+h of
// each set p; the layer-3 output of set p lands in one of the group's two 128-column regions,
// alternately, so the MMAs of set p+1 run during the splines of set p.  Every wait on the tensor
// cores is bounded; on a timeout the kernel records it in the status word, still waits (bounded)
// for all its MMAs, frees its TMEM and returns.
namespace umma {

constexpr int kTile = 128;          // events per tile (TMEM lanes)
constexpr int kGroupThreads = 256;  // one tile in flight per group of two warpgroups
constexpr int kInFlight = 2;        // groups (tiles in flight) per CTA
constexpr int kThreads = kGroupThreads * kInFlight;
constexpr int kQRowsU = 56;         // W3 rows per transformed dim in shared memory (3K+1 = 49 used)
constexpr int kTmemCols = 512;      // group g owns [256g, 256g + 256): two regions of 128 columns

// Shared memory: the weights, then per group an input tile and an activation tile, the biases and
// the log-det hand-over.  W3 holds the nb transformed dims (each dim's rows in the interleaved
// order of locate_pairs, so that a width and its height leave the MMA as a register pair, and
// the layer-3 biases likewise) at a stride of 56 rows plus 8 zero
// rows, so that the 64-row B operand of the last dim stays inside it (its rows 49..63 only feed
// output columns that are never read).
struct Smem {
    static constexpr size_t w1 = 0;                          // 128 x 16 bf16
    static constexpr size_t w2 = w1 + 128 * kInPad * 2;      // 128 x 128
    static constexpr size_t w3 = w2 + 128 * 128 * 2;         // (nb x 56 + 8) x 128
    static constexpr size_t in_bytes = kTile * kInPad * 2;
    static constexpr size_t act_bytes = kTile * 128 * 2;
    static constexpr size_t tail_bytes = (128 + 128 + 8 * 56 + kInFlight * kTile) * 4;
    __host__ __device__ static constexpr size_t w3_bytes(int nb) { return static_cast<size_t>(nb * kQRowsU + 8) * 128 * 2; }
    __host__ __device__ static constexpr size_t in(int nb) { return w3 + w3_bytes(nb); }
    __host__ __device__ static constexpr size_t act(int nb) { return in(nb) + kInFlight * in_bytes; }
    __host__ __device__ static constexpr size_t tail(int nb) { return act(nb) + kInFlight * act_bytes; }
    __host__ __device__ static constexpr size_t total(int nb) { return tail(nb) + tail_bytes; }
};
static_assert(Smem::total(kMaxNb) <= 232448, "the tcgen05 layer must fit the 227 KB of shared memory of a CTA");

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// element offset of (row, k) in a [rows][K] K-major canonical tile
__device__ __forceinline__ int coff(int row, int k, int K) {
    return (((row >> 3) * (K >> 3) + (k >> 3)) * 8 + (row & 7)) * 8 + (k & 7);
}

// shared-memory matrix descriptor: start, leading (K-direction) and stride (row-direction)
// byte offsets between core matrices, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((addr >> 4) & 0x3FFF) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32) | (static_cast<uint64_t>(1) << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M = 128
__device__ __forceinline__ uint32_t idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(128 >> 4) << 24);
}

// D[tmem] (+)= A[128 x K] B[n x K]^T over K in steps of 16 (one thread)
__device__ __forceinline__ void mma_chain(uint32_t tmem, uint32_t a_addr, uint32_t b_addr, int K, int n) {
    const uint32_t sbo = (K / 8) * 128, id = idesc(n);
    for (int s = 0; s < K / 16; ++s) {
        const uint64_t ad = sdesc(a_addr + s * 256, 128, sbo), bd = sdesc(b_addr + s * 256, 128, sbo);
        const uint32_t acc = s > 0 ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc));
    }
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(mbar)));
}

constexpr int kWaitPolls = 1 << 24;  // default bound of a completion wait (polls of try_wait)

// bounded wait for the given phase of the mbarrier; false on timeout
__device__ __forceinline__ bool wait_phase(uint64_t* mbar, uint32_t phase, int limit) {
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(su32(mbar)), "r"(phase));
        if (done) return true;
    }
    return false;
}

#define PS_TMEM_LD32(v, addr)                                                                                   \
    asm volatile(                                                                                               \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17," \
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"                                    \
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),       \
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), \
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),            \
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),            \
          "=r"(v[30]), "=r"(v[31])                                                                            \
        : "r"(addr))
#define PS_TMEM_LD16(v, addr)                                                                                   \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, " \
                 "[%16];\n"                                                                                     \
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), \
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),      \
                   "=r"(v[15])                                                                                  \
                 : "r"(addr))
#define PS_TMEM_LD8(v, addr)                                                                                    \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"                     \
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]) \
                 : "r"(addr))

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// SiLU of two hidden columns, z / (1 + 2^(-z log2 e)) with z = acc + bias, in paired FP32
// arithmetic (one instruction per pair for the adds and multiplies, each exactly rounded like
// its scalar form) and the hardware exponential and reciprocal, as bfloat16x2.  For z -> -inf
// the denominator overflows and the result is 0.
__device__ __forceinline__ uint32_t silu_pair_bf16(float a0, float a1, float c0, float c1, float2& z) {
    z = __fadd2_rn(make_float2(a0, a1), make_float2(c0, c1));
    const float2 t = __fmul2_rn(z, make_float2(-kLog2e, -kLog2e));
    const float2 den = __fadd2_rn(make_float2(ex2_approx(t.x), ex2_approx(t.y)), make_float2(1.0f, 1.0f));
    const float2 y = __fmul2_rn(z, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
    return pack_bf16(y.x, y.y);
}

// 32 hidden columns of this thread's event: + bias, SiLU, bf16 into the operand tile; for training
// (kStore) also the pre-activations z (FP32) and the activations (bf16) into this event's rows zg,
// ag where `store` holds.  The TMEM load is warp-collective (.sync.aligned): every lane of the warp
// executes it, whatever `store` is.
template <bool kStore>
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, const float* bias, bf16* act, int row, int c0,
                                                bool store = false, float* zg = nullptr, bf16* ag = nullptr) {
    uint32_t v[32];
    __syncwarp();  // the warp-collective TMEM load is issued by a converged warp
    PS_TMEM_LD32(v, taddr + c0);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const float4 b0 = *reinterpret_cast<const float4*>(bias + c0 + j);
        const float4 b1v = *reinterpret_cast<const float4*>(bias + c0 + j + 4);
        uint4 o;
        float2 z0, z1, z2, z3;
        o.x = silu_pair_bf16(__uint_as_float(v[j]), __uint_as_float(v[j + 1]), b0.x, b0.y, z0);
        o.y = silu_pair_bf16(__uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]), b0.z, b0.w, z1);
        o.z = silu_pair_bf16(__uint_as_float(v[j + 4]), __uint_as_float(v[j + 5]), b1v.x, b1v.y, z2);
        o.w = silu_pair_bf16(__uint_as_float(v[j + 6]), __uint_as_float(v[j + 7]), b1v.z, b1v.w, z3);
        *reinterpret_cast<uint4*>(act + coff(row, c0 + j, 128)) = o;
        if (kStore && store) {
            *reinterpret_cast<float4*>(zg + c0 + j) = make_float4(z0.x, z0.y, z1.x, z1.y);
            *reinterpret_cast<float4*>(zg + c0 + j + 4) = make_float4(z2.x, z2.y, z3.x, z3.y);
            *reinterpret_cast<uint4*>(ag + c0 + j) = o;
        }
    }
}

// The bin of v and what the forward and inverse bin formulas need, from raw parameters held in
// registers (compile-time indices only) in the interleaved order of the fused layer: width i at
// 2i, height i at 2i + 1 (i < K), knot derivatives at 2K..3K.  Widths and heights are handled as
// pairs in paired FP32 arithmetic, softmax exponentials as 2^(a log2 e - max log2 e).
struct BinF {
    float x0, y0, w, h, d0, d1;
};

// Position in that interleaved order of spline parameter p (widths 0..K-1, heights K..2K-1,
// derivatives 2K..3K), and the parameter at position j.
__host__ __device__ constexpr int il_pos(int p, int K) { return p < K ? 2 * p : p < 2 * K ? 2 * (p - K) + 1 : p; }
__host__ __device__ constexpr int il_param(int j, int K) { return j < 2 * K ? ((j & 1) ? K + (j >> 1) : (j >> 1)) : j; }

template <int K>
__device__ __forceinline__ BinF locate_pairs(const float (&raw)[3 * K + 1], float v, bool by_height) {
    static_assert((K & (K - 1)) == 0, "pairwise maxima need a power-of-two bin count");
    // the maxima by a tree (a maximum is exact in any order)
    float mxw[K], mxh[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        mxw[i] = raw[2 * i];
        mxh[i] = raw[2 * i + 1];
    }
#pragma unroll
    for (int s = K / 2; s > 0; s >>= 1)
#pragma unroll
        for (int i = 0; i < s; ++i) {
            mxw[i] = fmaxf(mxw[i], mxw[i + s]);
            mxh[i] = fmaxf(mxh[i], mxh[i + s]);
        }
    const float mw = mxw[0], mh = mxh[0];
    const float2 l2e = make_float2(kLog2e, kLog2e), nm = make_float2(-mw * kLog2e, -mh * kLog2e);
    float2 e[K];
    float2 z = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const float2 t = __ffma2_rn(make_float2(raw[2 * i], raw[2 * i + 1]), l2e, nm);
        e[i] = make_float2(ex2_approx(t.x), ex2_approx(t.y));
        z = __fadd2_rn(z, e[i]);
    }
    const float2 iz = make_float2(rcp_approx(z.x), rcp_approx(z.y));
    const float2 c = make_float2(1.0f - K * kMinW, 1.0f - K * kMinH), mins = make_float2(kMinW, kMinH);
    // The bin is the first i with v below its right edge (the last bin otherwise).  The edges rise
    // strictly (every width is at least kMinW), so s_i = [v < edge_i] steps once from 0 to 1 and
    // hit_i = s_i - s_(i-1) is 1 for that bin alone.  Its values are gathered without branches as
    // sums of hit_i x value: a multiply by 0 or 1 and an add of +0 are exact, so the gathered
    // values are the bin's own, bit for bit.
    float2 lo = make_float2(0.0f, 0.0f), wh_sel = make_float2(0.0f, 0.0f);
    float a0 = 0.0f, a1 = 0.0f;
    float2 cum = make_float2(0.0f, 0.0f);
    float prev = 0.0f;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const float2 wh = __ffma2_rn(c, __fmul2_rn(e[i], iz), mins);  // (width, height) of bin i
        const float2 next = __fadd2_rn(cum, wh);
        const float s = (i == K - 1 || (by_height ? v < next.y : v < next.x)) ? 1.0f : 0.0f;
        const float hit = s - prev;
        const float2 hh = make_float2(hit, hit);
        lo = __ffma2_rn(hh, cum, lo);
        wh_sel = __ffma2_rn(hh, wh, wh_sel);
        a0 = __fmaf_rn(hit, raw[2 * K + i], a0);
        a1 = __fmaf_rn(hit, raw[2 * K + i + 1], a1);
        prev = s;
        cum = next;
    }
    BinF b;
    b.x0 = lo.x;
    b.y0 = lo.y;
    b.w = wh_sel.x;
    b.h = wh_sel.y;
    b.d0 = kMinD + softplus(a0);
    b.d1 = kMinD + softplus(a1);
    return b;
}

__device__ __forceinline__ void group_sync(int grp) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(1 + grp), "r"(kGroupThreads) : "memory");
}

// layer 3 of transformed dims 2p and 2p+1 (those below nb): one N = 64 chain each, B from row 56q
// of W3, into columns 0 and 64 of the region
__device__ __forceinline__ void issue_set(uint32_t region, uint32_t act_addr, uint32_t w3_addr, int p, int nb) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int q = 2 * p + u;
        if (q < nb) mma_chain(region + 64 * u, act_addr, w3_addr + q * (kQRowsU / 8) * 2048, 128, 64);
    }
}

// What the training forward keeps for the backward pass (row-major per event unless stated):
// the bf16 MLP input In [B][16], pre-activations Z1, Z2 (FP32) and activations A1, A2 (bf16)
// [B][128], the raw spline parameters P parameter-major [q (3K+1) + j][ldp], and the next
// layer's state Xn [B][d] (X itself is left unchanged).
struct TrainOut {
    bf16* In;
    float* Z1;
    float* Z2;
    bf16* A1;
    bf16* A2;
    float* P;
    int64_t ldp;
    float* Xn;
};

template <bool kInverse, bool kTrain>
__global__ void __launch_bounds__(kThreads, 1)
    k_layer_umma(int64_t B, int d, float* X, float* logdet, const __grid_constant__ LayerDesc ld, const bf16* W1,
                 const float* b1, const bf16* W2, const float* b2, const bf16* W3, const float* b3,
                 unsigned long long* status, int wait_limit, int debug_flags, const __grid_constant__ TrainOut tr) {
    static_assert(!(kInverse && kTrain), "the training forward runs the forward direction");
    constexpr int K = 16, PQ = 3 * K + 1;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nb = ld.nb;
    bf16* w1s = reinterpret_cast<bf16*>(smem + Smem::w1);
    bf16* w2s = reinterpret_cast<bf16*>(smem + Smem::w2);
    bf16* w3s = reinterpret_cast<bf16*>(smem + Smem::w3);
    float* b1s = reinterpret_cast<float*>(smem + Smem::tail(nb));
    float* b2s = b1s + 128;
    float* b3s = b2s + 128;
    float* lds = b3s + 8 * 56;  // log-det hand-over, [group][row]
    __shared__ __align__(8) uint64_t mbar[kInFlight][2];  // per group: L1, L2, even sets | odd sets
    __shared__ __align__(8) uint64_t drain;               // end-of-kernel completion of every MMA issued
    __shared__ uint32_t tmem_holder;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = tid / kGroupThreads;          // the group (tile slot) of this thread
    const int h = (warp >> 2) & 1;                // warpgroup within the group
    const int row = 32 * (warp & 3) + lane;       // this thread's event in the tile (TMEM lane)
    const bool issuer = (tid % kGroupThreads) == 0;
    bf16* ins = reinterpret_cast<bf16*>(smem + Smem::in(nb) + grp * Smem::in_bytes);
    bf16* act = reinterpret_cast<bf16*>(smem + Smem::act(nb) + grp * Smem::act_bytes);
    const int nsets = (nb + 1) / 2;

    // weights into the canonical layout, 8 consecutive k (one core-matrix row) per 16-byte copy
    for (int i = tid; i < 128 * kInPad / 8; i += kThreads) {
        const int r = i / (kInPad / 8), k = (i % (kInPad / 8)) * 8;
        *reinterpret_cast<uint4*>(w1s + coff(r, k, kInPad)) = *reinterpret_cast<const uint4*>(W1 + r * kInPad + k);
    }
    for (int i = tid; i < 128 * 16; i += kThreads) {
        const int r = i >> 4, k = (i & 15) * 8;
        *reinterpret_cast<uint4*>(w2s + coff(r, k, 128)) = *reinterpret_cast<const uint4*>(W2 + r * 128 + k);
    }
    for (int i = tid; i < (nb * kQRowsU + 8) * 16; i += kThreads) {
        const int r = i >> 4, k = (i & 15) * 8;
        const int q = r / kQRowsU, j = r % kQRowsU;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (q < nb && j < PQ) v = *reinterpret_cast<const uint4*>(W3 + (q * PQ + il_param(j, K)) * 128 + k);
        *reinterpret_cast<uint4*>(w3s + coff(r, k, 128)) = v;
    }
    for (int i = tid; i < 128; i += kThreads) {
        b1s[i] = b1[i];
        b2s[i] = b2[i];
    }
    for (int i = tid; i < 8 * 56; i += kThreads) {
        const int q = i / 56, j = i % 56;
        b3s[i] = (q < nb && j < PQ) ? b3[q * PQ + il_param(j, K)] : 0.0f;
    }
    if (tid == 0) {
        failed = 0;
        for (int g = 0; g < kInFlight; ++g)
            for (int k = 0; k < 2; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&mbar[g][k])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(&drain)), "r"(kInFlight));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_holder)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tg = tmem_holder + 256 * grp;                                 // this group's columns
    const uint32_t tlane = tg + (static_cast<uint32_t>(32 * (warp & 3)) << 16);  // this warp's TMEM lanes
    uint32_t phase = 0u;  // bit k: the parity this thread waits for next on completion barrier k
    // one bounded wait on barrier k of this group
    auto wait_on = [&](int k) {
        if (!wait_phase(&mbar[grp][k], (phase >> k) & 1u, wait_limit)) failed = 1;
        phase ^= 1u << k;
        fence_after();
    };

    const int64_t n_tiles = (B + kTile - 1) / kTile;
    const int64_t first = 2 * static_cast<int64_t>(blockIdx.x) + grp;
    const int64_t stride = kInFlight * static_cast<int64_t>(gridDim.x);
    // the conditioning dims of the tile (warpgroup h: k = 8h .. 8h+7), loaded one tile ahead so that
    // the loads overlap the previous tile's work
    float cond[8];
    auto load_cond = [&](int64_t t) {
        const int64_t e = t * kTile + row;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = 8 * h + i;
            cond[i] = (e < B && k < ld.na) ? X[e * d + ld.ta[k]] : 0.0f;
        }
    };
    load_cond(first);
    for (int64_t tile = first; tile < n_tiles; tile += stride) {
        const int64_t ev = tile * kTile + row;
        const bool valid = ev < B;
        // this thread's transformed dims (2p + h of set p), loaded now so that the loads overlap the
        // MLP rather than stall the splines
        float xq[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int q = 2 * p + h;
            xq[p] = (valid && q < nb) ? X[ev * d + ld.tb[q]] : 0.0f;
        }
        // operand tile of the conditioning dims, then the next tile's conditioning dims
        {
            uint4 o;
            o.x = pack_bf16(cond[0], cond[1]);
            o.y = pack_bf16(cond[2], cond[3]);
            o.z = pack_bf16(cond[4], cond[5]);
            o.w = pack_bf16(cond[6], cond[7]);
            *reinterpret_cast<uint4*>(ins + coff(row, 8 * h, kInPad)) = o;
            if constexpr (kTrain) {  // the MLP input, and the conditioning dims carried into Xn
                if (valid) {
                    *reinterpret_cast<uint4*>(tr.In + ev * kInPad + 8 * h) = o;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (8 * h + i < ld.na) tr.Xn[ev * d + ld.ta[8 * h + i]] = cond[i];
                }
            }
        }
        load_cond(tile + stride);
        // layer 1
        fence_async_smem();
        fence_before();
        group_sync(grp);
        if (issuer) {
            fence_after();
            mma_chain(tg, su32(ins), su32(w1s), kInPad, 128);
            // test flag: withhold the group's first completion signal, so that the wait runs out
            if (!((debug_flags & 1) && tile == first)) commit(&mbar[grp][0]);
        }
        wait_on(0);
        {  // warp-uniform calls: the stores are predicated per lane inside
            float* zg = kTrain ? tr.Z1 + ev * 128 : nullptr;
            bf16* ag = kTrain ? tr.A1 + ev * 128 : nullptr;
            hidden_epilogue<kTrain>(tlane, b1s, act, row, 64 * h, valid, zg, ag);
            hidden_epilogue<kTrain>(tlane, b1s, act, row, 64 * h + 32, valid, zg, ag);
        }
        // layer 2
        fence_async_smem();
        fence_before();
        group_sync(grp);
        if (issuer) {
            fence_after();
            mma_chain(tg, su32(act), su32(w2s), 128, 128);
            commit(&mbar[grp][0]);
        }
        wait_on(0);
        {  // layer-2 reads of act are complete; warp-uniform calls as above
            float* zg = kTrain ? tr.Z2 + ev * 128 : nullptr;
            bf16* ag = kTrain ? tr.A2 + ev * 128 : nullptr;
            hidden_epilogue<kTrain>(tlane, b2s, act, row, 64 * h, valid, zg, ag);
            hidden_epilogue<kTrain>(tlane, b2s, act, row, 64 * h + 32, valid, zg, ag);
        }
        fence_async_smem();
        fence_before();
        group_sync(grp);
        // layer 3 and the splines, set p = dims 2p, 2p+1 in region 128 (p even) or 0 (p odd) of the
        // group; completions alternate between the group's two barriers, so a wait can never see
        // a later completion on its barrier before every thread has passed the group barrier
        float lsum = 0.0f;
        if (issuer) {
            fence_after();
            issue_set(tg + 128, su32(act), su32(w3s), 0, nb);
            commit(&mbar[grp][0]);
        }
        for (int p = 0; p < nsets; ++p) {
            wait_on(p & 1);
            const int q = 2 * p + h;
            float raw[PQ];
            {
                uint32_t v[56];
                const uint32_t a = tlane + ((p & 1) ? 0 : 128) + 64 * h;  // column-aligned loads
                __syncwarp();
                PS_TMEM_LD32(v, a);
                uint32_t* v2 = v + 32;
                PS_TMEM_LD16(v2, a + 32);
                uint32_t* v3 = v + 48;
                PS_TMEM_LD8(v3, a + 48);
                tmem_wait_ld();
                // the biases four at a time (row 56q of b3s is 16-byte aligned), added in pairs
                const float* bq = b3s + (q < 8 ? q * 56 : 0);
#pragma unroll
                for (int j = 0; j + 3 < PQ; j += 4) {
                    const float4 b = *reinterpret_cast<const float4*>(bq + j);
                    const float2 t0 = __fadd2_rn(make_float2(__uint_as_float(v[j]), __uint_as_float(v[j + 1])),
                                                 make_float2(b.x, b.y));
                    const float2 t1 = __fadd2_rn(make_float2(__uint_as_float(v[j + 2]), __uint_as_float(v[j + 3])),
                                                 make_float2(b.z, b.w));
                    raw[j] = t0.x;
                    raw[j + 1] = t0.y;
                    raw[j + 2] = t1.x;
                    raw[j + 3] = t1.y;
                }
                raw[PQ - 1] = __uint_as_float(v[PQ - 1]) + bq[PQ - 1];
            }
            // the other region was read completely before the previous group barrier
            if (issuer && p + 1 < nsets) {
                fence_after();
                issue_set(tg + ((p & 1) ? 128 : 0), su32(act), su32(w3s), p + 1, nb);
                commit(&mbar[grp][(p + 1) & 1]);
            }
            if constexpr (kTrain) {  // the raw spline parameters, parameter-major
                if (valid && q < nb)
#pragma unroll
                    for (int j = 0; j < PQ; ++j)
                        tr.P[static_cast<int64_t>(q * PQ + j) * tr.ldp + ev] = raw[il_pos(j, K)];
            }
            if (valid && q < nb) {
                const int jd = ld.tb[q];
                const float xv = fminf(fmaxf(p == 0 ? xq[0] : p == 1 ? xq[1] : p == 2 ? xq[2] : xq[3], 0.0f), 1.0f);
                const BinF bn = locate_pairs<K>(raw, xv, kInverse);
                float F, Fp;
                if (!kInverse) {
                    bin_eval<float>(xv, bn.x0, bn.w, bn.y0, bn.h, bn.d0, bn.d1, F, Fp);
                    (kTrain ? tr.Xn : X)[ev * d + jd] = fminf(fmaxf(F, 1e-7f), 1.0f - 1e-7f);
                    lsum += __logf(Fp);
                } else {
                    const float sl = bn.h / bn.w, dy = xv - bn.y0, e = bn.d1 + bn.d0 - 2.0f * sl;
                    const float qa = bn.h * (sl - bn.d0) + dy * e, qb = bn.h * bn.d0 - dy * e, qc = -sl * dy;
                    const float disc = fmaxf(qb * qb - 4.0f * qa * qc, 0.0f);
                    const float den = -qb - sqrtf(disc);
                    const float xi = den != 0.0f ? fminf(fmaxf(2.0f * qc / den, 0.0f), 1.0f) : 0.0f;
                    const float x = bn.x0 + xi * bn.w;
                    bin_eval<float>(x, bn.x0, bn.w, bn.y0, bn.h, bn.d0, bn.d1, F, Fp);
                    X[ev * d + jd] = fminf(fmaxf(x, 0.0f), 1.0f);
                    lsum -= __logf(Fp);
                }
            }
            fence_before();
            group_sync(grp);  // every thread's reads of this region precede the MMAs of set p+2
        }
        if (h == 1) lds[grp * kTile + row] = lsum;
        group_sync(grp);
        // a reduction in memory (no value returned, so nothing waits on the load); the only
        // update of this element in the launch, rounded as the plain add
        if (h == 0 && valid) atomicAdd(logdet + ev, lsum + lds[grp * kTile + row]);
    }
    // drain: after a wait that ran out, MMAs may still be in flight; the TMEM is freed only after a
    // commit issued by each group behind all of its MMAs has arrived (default bound)
    if (issuer) commit(&drain);
    if (!wait_phase(&drain, 0, kWaitPolls)) failed = 1;
    fence_after();
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_holder), "r"(kTmemCols));
    if (tid == 0 && failed) atomicAdd(status, 1ULL);
}

}  // namespace umma

// out[j ldr + col0 + b] <- X[b d + j] (event-major float -> SoA double)
__global__ void k_store_cols(int64_t B, int d, int64_t col0, int64_t ldr, const float* X, double* out) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b >= B) return;
    for (int j = 0; j < d; ++j) out[j * ldr + col0 + b] = static_cast<double>(X[b * d + j]);
}

__global__ void k_store_ld(int64_t B, int64_t col0, const float* ld, double* out) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b < B) out[col0 + b] = static_cast<double>(ld[b]);
}

// X[L] <- r (SoA double -> event-major float)
__global__ void k_load_r(int64_t B, int d, int64_t col0, int64_t ldr, const double* r, float* X) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b >= B) return;
    for (int j = 0; j < d; ++j) X[b * d + j] = static_cast<float>(r[j * ldr + col0 + b]);
}

// r (and optionally z) in the SoA layout of the phase-space map's explicit-input mode
__global__ void k_store_r(int64_t B, int d, int64_t col0, int64_t ldr, const float* X, const float* X0,
                          const float* logdet, double* r, double* ld_out, double* z) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b >= B) return;
    for (int j = 0; j < d; ++j) r[j * ldr + col0 + b] = static_cast<double>(X[b * d + j]);
    if (z)
        for (int j = 0; j < d; ++j) z[j * ldr + col0 + b] = static_cast<double>(X0[b * d + j]);
    if (ld_out) ld_out[col0 + b] = static_cast<double>(logdet[b]);
}

__global__ void k_combine(int64_t B, const double* wmap, const double* logdet, double* w) {
    int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b >= B) return;
    double v = wmap[b] * exp(logdet[b]);
    w[b] = isfinite(v) ? v : 0.0;
}

// Adam on the FP32 master parameters, then the bf16 copy
__global__ void k_adam(int64_t n, float* p, const float* g, float* m, float* v, bf16* pb, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    if (!isfinite(gi)) gi = 0.0f;
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16(pi);
}

__global__ void k_to_bf16(int64_t n, const float* p, bf16* pb) {
    int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16(p[i]);
}

}  // namespace flow
}  // namespace ps

// ===========================================================================================
// host side
using namespace ps::flow;

namespace {
thread_local std::string f_err;
int ffail(int code, const std::string& m) {
    f_err = m;
    return code;
}
int fcheck(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return PS_OK;
    return ffail(PS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
struct Guard {
    int prev = -1;
    explicit Guard(int d) {
        if (cudaGetDevice(&prev) == cudaSuccess) cudaSetDevice(d);
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
inline unsigned blocks(int64_t n, int t) { return static_cast<unsigned>((n + t - 1) / t); }
}  // namespace

struct ps_flow_s {
    FlowDesc fd;
    int device = 0;
    int sms = 1;
    int64_t max_batch = 0;
    int64_t n_params = 0;
    // parameters and optimiser state (device)
    float* p = nullptr;
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    bf16* pb = nullptr;
    int64_t step = 0;
    // activations of the last sampled batch
    int64_t batch = 0;
    float* X = nullptr;      // [L+1][max_batch][d]
    bf16* In = nullptr;      // [L][max_batch][16]
    float* Z1 = nullptr;     // [L][max_batch][H]
    float* Z2 = nullptr;
    bf16* A1 = nullptr;
    bf16* A2 = nullptr;
    float* Praw = nullptr;   // [L][Pmax][max_batch] (parameter-major)
    float* logdet = nullptr; // [max_batch]
    // backward scratch
    float* G = nullptr;      // [Pmax][max_batch]
    bf16* Gb = nullptr;
    float* dA = nullptr;     // [max_batch][H]
    float* dZ = nullptr;
    bf16* dZb = nullptr;
    bf16* dAb = nullptr;
    float* dIn = nullptr;    // [max_batch][16]
    float* gX = nullptr;     // [max_batch][d]
    float* gXn = nullptr;
    double* wtot = nullptr;  // [max_batch]
    double* scal = nullptr;  // [0] sum w, [1] loss
    int Pmax = 0;
    // buffers of the fused sampling / density path (allocated on first use)
    int64_t gen_cap = 0;
    float* gen_X = nullptr;   // [gen_cap][d]
    float* gen_ld = nullptr;  // [gen_cap]
    unsigned long long* gen_status = nullptr;  // tensor-core waits that timed out
    int wait_limit = umma::kWaitPolls;         // bound of every completion wait (polls)
    int debug_flags = 0;                       // tests only (ps_flow_set_debug)
};

namespace {

void free_flow(ps_flow f) {
    for (void* q : {static_cast<void*>(f->p), static_cast<void*>(f->grad), static_cast<void*>(f->m),
                    static_cast<void*>(f->v), static_cast<void*>(f->pb), static_cast<void*>(f->X),
                    static_cast<void*>(f->In), static_cast<void*>(f->Z1), static_cast<void*>(f->Z2),
                    static_cast<void*>(f->A1), static_cast<void*>(f->A2), static_cast<void*>(f->Praw),
                    static_cast<void*>(f->logdet), static_cast<void*>(f->G), static_cast<void*>(f->Gb),
                    static_cast<void*>(f->dA), static_cast<void*>(f->dZ), static_cast<void*>(f->dZb), static_cast<void*>(f->dAb),
                    static_cast<void*>(f->dIn), static_cast<void*>(f->gX), static_cast<void*>(f->gXn),
                    static_cast<void*>(f->wtot), static_cast<void*>(f->scal),
                    static_cast<void*>(f->gen_X), static_cast<void*>(f->gen_ld),
                    static_cast<void*>(f->gen_status)})
        cudaFree(q);
}

uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// launch one GEMM; kchunk = K unless split
int gemm(const GemmArgs& a0, int splits, cudaStream_t st) {
    GemmArgs a = a0;
    a.a_vec = (reinterpret_cast<uintptr_t>(a.A) & 15) == 0;
    a.b_vec = (reinterpret_cast<uintptr_t>(a.B) & 15) == 0;
    splits = std::max(1, splits);
    a.kchunk = ((a.K + splits - 1) / splits + 31) / 32 * 32;
    int nz = (a.K + a.kchunk - 1) / a.kchunk;
    dim3 grid((a.M + 63) / 64, (a.N + 63) / 64, nz);
    k_gemm<<<grid, 128, 0, st>>>(a);
    ps::count_launches(1);
    return fcheck(cudaGetLastError(), "k_gemm");
}

// One backward GEMM on bwg::k_gemm_bw: false (nothing launched) when the operands break the
// 16-byte rules of its cp.async copies (tensor starts aligned, row strides multiples of 8
// elements), in which case the caller takes k_gemm.
bool gemm_bw_fits(const bwg::Args& a, bool am) {
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    return al(a.A) && al(a.B) && (am ? a.lak : a.lam) % 8 == 0 && a.ldb % 8 == 0;
}
bool gemm_bw(bwg::Args a, bool am, int epi, int splits, cudaStream_t st, int* status) {
    auto al = [](const void* p, uintptr_t m) { return (reinterpret_cast<uintptr_t>(p) & m) == 0; };
    if (!gemm_bw_fits(a, am)) return false;
    const bool narrow = a.N <= 16;
    splits = std::max(1, splits);
    a.kchunk = std::max(32, ((a.K + splits - 1) / splits + 31) / 32 * 32);
    const int nz = std::max(1, (a.K + a.kchunk - 1) / a.kchunk);
    const int bn = narrow ? 16 : 128;
    const dim3 grid((a.M + bwg::kBM - 1) / bwg::kBM, (a.N + bn - 1) / bn, nz);
    int pairs = 0;
    if (epi == bwg::kStore) pairs = al(a.C, 7) && a.ldc % 2 == 0;
    if (epi == bwg::kSiluGrad) pairs = al(a.Zs, 7) && a.ldz % 2 == 0 && al(a.Cb, 3) && a.ldcb % 2 == 0;
    const size_t smem = bwg::smem_bytes(bn);
    const int key = (narrow ? 100 : 0) + (am ? 10 : 0) + epi;
    switch (key) {
        case 0 + bwg::kAtomic: bwg::k_gemm_bw<128, false, bwg::kAtomic><<<grid, bwg::kThreads, smem, st>>>(a, pairs); break;
        case 0 + bwg::kSiluGrad: bwg::k_gemm_bw<128, false, bwg::kSiluGrad><<<grid, bwg::kThreads, smem, st>>>(a, pairs); break;
        case 10 + bwg::kAtomic: bwg::k_gemm_bw<128, true, bwg::kAtomic><<<grid, bwg::kThreads, smem, st>>>(a, pairs); break;
        case 10 + bwg::kSiluGrad: bwg::k_gemm_bw<128, true, bwg::kSiluGrad><<<grid, bwg::kThreads, smem, st>>>(a, pairs); break;
        case 110 + bwg::kAtomic: bwg::k_gemm_bw<16, true, bwg::kAtomic><<<grid, bwg::kThreads, smem, st>>>(a, pairs); break;
        case 100 + bwg::kStore: bwg::k_gemm_bw<16, false, bwg::kStore><<<grid, bwg::kThreads, smem, st>>>(a, pairs); break;
        default: return false;  // a shape the backward pass does not use
    }
    ps::count_launches(1);
    *status = fcheck(cudaGetLastError(), "k_gemm_bw");
    return true;
}

// MLP of layer l on the conditioning dims of Xl (activations kept for the backward pass)
int mlp(ps_flow f, int l, int64_t B, const float* Xl, cudaStream_t st) {
    const FlowDesc& fd = f->fd;
    const int d = fd.d, H = fd.H, T = 256;
    {
        const LayerDesc& ld = fd.layer[l];
        bf16* In = f->In + static_cast<int64_t>(l) * f->max_batch * kInPad;
        float* Z1 = f->Z1 + static_cast<int64_t>(l) * f->max_batch * H;
        float* Z2 = f->Z2 + static_cast<int64_t>(l) * f->max_batch * H;
        bf16* A1 = f->A1 + static_cast<int64_t>(l) * f->max_batch * H;
        bf16* A2 = f->A2 + static_cast<int64_t>(l) * f->max_batch * H;
        float* P = f->Praw + static_cast<int64_t>(l) * f->max_batch * f->Pmax;
        k_gather<<<blocks(B, T), T, 0, st>>>(B, d, Xl, ld, In);
        int s;
        GemmArgs g{};
        g.A = In; g.lam = kInPad; g.lak = 1; g.B = f->pb + ld.off_W1; g.lbn = kInPad; g.lbk = 1;
        g.M = static_cast<int>(B); g.N = H; g.K = kInPad; g.bias = f->p + ld.off_b1; g.C = Z1; g.ldc = H; g.Cb = A1;
        g.ldcb = H; g.act = 1;
        s = gemm(g, 1, st);
        if (s != PS_OK) return s;
        g = GemmArgs{};
        g.A = A1; g.lam = H; g.lak = 1; g.B = f->pb + ld.off_W2; g.lbn = H; g.lbk = 1;
        g.M = static_cast<int>(B); g.N = H; g.K = H; g.bias = f->p + ld.off_b2; g.C = Z2; g.ldc = H; g.Cb = A2;
        g.ldcb = H; g.act = 1;
        s = gemm(g, 1, st);
        if (s != PS_OK) return s;
        g = GemmArgs{};
        g.A = A2; g.lam = H; g.lak = 1; g.B = f->pb + ld.off_W3; g.lbn = H; g.lbk = 1;
        g.M = static_cast<int>(B); g.N = ld.Ppad; g.K = H; g.bias = f->p + ld.off_b3; g.C = P; g.ldc = f->max_batch;
        g.trans_c = 1;
        s = gemm(g, 1, st);
        if (s != PS_OK) return s;
    }
    ps::count_launches(1);
    return PS_OK;
}

// forward of all layers for a chunk of `B` events starting at event ev0; stores activations
bool fused_ok(const FlowDesc& fd);
int ensure_gen(ps_flow f);

int forward(ps_flow f, int64_t B, uint64_t seed, uint64_t ev0, cudaStream_t st) {
    const FlowDesc& fd = f->fd;
    const int d = fd.d, T = 256;
    k_init_z<<<blocks(B, T), T, 0, st>>>(B, d, seed, ev0, f->X);
    cudaMemsetAsync(f->logdet, 0, B * sizeof(float), st);
    if (fd.K == 16 && fused_ok(fd) && !(f->debug_flags & 2)) {
        // the tcgen05 layer in its training form: one launch per layer writes what the backward
        // pass reads (MLP input, pre-activations, activations, raw spline parameters, next state)
        int s = ensure_gen(f);
        if (s != PS_OK) return s;
        const int64_t tiles = (B + umma::kTile - 1) / umma::kTile;
        const unsigned grid =
            static_cast<unsigned>(std::min<int64_t>(f->sms, (tiles + umma::kInFlight - 1) / umma::kInFlight));
        for (int l = 0; l < fd.L; ++l) {
            const LayerDesc& lay = fd.layer[l];
            float* Xl = f->X + static_cast<int64_t>(l) * f->max_batch * d;
            umma::TrainOut tr;
            tr.In = f->In + static_cast<int64_t>(l) * f->max_batch * kInPad;
            tr.Z1 = f->Z1 + static_cast<int64_t>(l) * f->max_batch * fd.H;
            tr.Z2 = f->Z2 + static_cast<int64_t>(l) * f->max_batch * fd.H;
            tr.A1 = f->A1 + static_cast<int64_t>(l) * f->max_batch * fd.H;
            tr.A2 = f->A2 + static_cast<int64_t>(l) * f->max_batch * fd.H;
            tr.P = f->Praw + static_cast<int64_t>(l) * f->max_batch * f->Pmax;
            tr.ldp = f->max_batch;
            tr.Xn = Xl + f->max_batch * d;
            umma::k_layer_umma<false, true><<<grid, umma::kThreads, umma::Smem::total(lay.nb), st>>>(
                B, d, Xl, f->logdet, lay, f->pb + lay.off_W1, f->p + lay.off_b1, f->pb + lay.off_W2,
                f->p + lay.off_b2, f->pb + lay.off_W3, f->p + lay.off_b3, f->gen_status, f->wait_limit,
                f->debug_flags & 1, tr);
        }
        ps::count_launches(1 + fd.L);
        return fcheck(cudaGetLastError(), "flow forward (tcgen05)");
    }
    for (int l = 0; l < fd.L; ++l) {
        const LayerDesc& ld = fd.layer[l];
        float* Xl = f->X + static_cast<int64_t>(l) * f->max_batch * d;
        float* Xn = Xl + f->max_batch * d;
        int s = mlp(f, l, B, Xl, st);
        if (s != PS_OK) return s;
        const float* P = f->Praw + static_cast<int64_t>(l) * f->max_batch * f->Pmax;
        auto kf = fd.K == 16 ? k_spline_forward<16> : k_spline_forward<0>;
        kf<<<blocks(B, T), T, 0, st>>>(B, d, fd.K, Xl, Xn, P, f->max_batch, ld, f->logdet);
    }
    ps::count_launches(1 + fd.L);
    return fcheck(cudaGetLastError(), "flow forward");
}

// inverse of all layers for a chunk: X[L] (already loaded) -> X[0]; f->logdet receives log g
int inverse(ps_flow f, int64_t B, cudaStream_t st) {
    const FlowDesc& fd = f->fd;
    const int d = fd.d, T = 256;
    cudaMemsetAsync(f->logdet, 0, B * sizeof(float), st);
    for (int l = fd.L - 1; l >= 0; --l) {
        const LayerDesc& ld = fd.layer[l];
        float* Xl = f->X + static_cast<int64_t>(l) * f->max_batch * d;
        float* Xn = Xl + f->max_batch * d;
        // the conditioning dims of x^(l+1) equal those of x^(l)
        int s = mlp(f, l, B, Xn, st);
        if (s != PS_OK) return s;
        const float* P = f->Praw + static_cast<int64_t>(l) * f->max_batch * f->Pmax;
        auto ki = fd.K == 16 ? k_spline_inverse<16> : k_spline_inverse<0>;
        ki<<<blocks(B, T), T, 0, st>>>(B, d, fd.K, Xn, Xl, P, f->max_batch, ld, f->logdet);
    }
    ps::count_launches(fd.L);
    return fcheck(cudaGetLastError(), "flow inverse");
}

// backward sweep (layers 0 .. L-1) of the importance-weighted forward KL; accumulates f->grad
int backward(ps_flow f, int64_t B, cudaStream_t st) {
    const FlowDesc& fd = f->fd;
    const int d = fd.d, H = fd.H, T = 256;
    cudaMemsetAsync(f->gX, 0, B * d * sizeof(float), st);
    cudaMemsetAsync(f->grad, 0, f->n_params * sizeof(float), st);
    int launches = 0;
    const unsigned colsum_rows = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(512, B / 64)));
    // batch-long weight-gradient GEMMs: split the batch so that about two CTAs per SM run,
    // with at least 256 events per split
    auto split_for = [&](int M, int N) {
        const int64_t tiles = static_cast<int64_t>((M + 63) / 64) * ((N + 63) / 64);
        const int64_t want = (2 * f->sms + tiles - 1) / tiles;
        return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, B / 256)));
    };
    // the same for the 128 x 128 (or 128 x 16) tiles of k_gemm_bw
    auto split_bw = [&](int M, int N) {
        const int64_t tiles = static_cast<int64_t>((M + 127) / 128) * (N <= 16 ? 1 : (N + 127) / 128);
        const int64_t want = (2 * f->sms + tiles - 1) / tiles;
        return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, B / 256)));
    };
    for (int l = 0; l < fd.L; ++l) {
        const LayerDesc& ld = fd.layer[l];
        float* Xl = f->X + static_cast<int64_t>(l) * f->max_batch * d;
        bf16* In = f->In + static_cast<int64_t>(l) * f->max_batch * kInPad;
        float* Z1 = f->Z1 + static_cast<int64_t>(l) * f->max_batch * H;
        float* Z2 = f->Z2 + static_cast<int64_t>(l) * f->max_batch * H;
        bf16* A1 = f->A1 + static_cast<int64_t>(l) * f->max_batch * H;
        bf16* A2 = f->A2 + static_cast<int64_t>(l) * f->max_batch * H;
        float* P = f->Praw + static_cast<int64_t>(l) * f->max_batch * f->Pmax;
        const int64_t ldg = f->max_batch;  // G, Gb and Praw are parameter-major
        // last linear layer: dW3 += G^T A2, db3 += rowsum G, dA2 = G W3 and its SiLU' form.  The
        // fast GEMM sums the rows of the BF16 adjoint itself; the fallback needs its FP32 copy.
        const int Bi = static_cast<int>(B);
        int s = PS_OK;
        bwg::Args w{};
        w.A = f->Gb; w.lam = ldg; w.lak = 1; w.B = A2; w.ldb = H;
        w.M = ld.Ppad; w.N = H; w.K = Bi; w.C = f->grad + ld.off_W3; w.ldc = H; w.rowsum = f->grad + ld.off_b3;
        const bool fast3 = gemm_bw_fits(w, false);
        auto kb = fd.K == 16 ? k_spline_backward<16> : k_spline_backward<0>;
        kb<<<blocks(B, T), T, 0, st>>>(B, d, fd.K, Xl, P, ldg, ld, f->gX, f->wtot, f->scal, fast3 ? nullptr : f->G,
                                       f->Gb, f->gXn, f->scal + 1);
        if (!fast3 || !gemm_bw(w, false, bwg::kAtomic, split_bw(ld.Ppad, H), st, &s)) {
            k_rowsum<<<dim3(std::min<unsigned>(blocks(B, 256), 4), ld.Ppad), 256, 0, st>>>(B, ldg, f->G,
                                                                                             f->grad + ld.off_b3);
            launches += 1;
            GemmArgs g{};
            g.A = f->Gb; g.lam = ldg; g.lak = 1; g.B = A2; g.lbn = 1; g.lbk = H;
            g.M = ld.Ppad; g.N = H; g.K = Bi; g.C = f->grad + ld.off_W3; g.ldc = H; g.atomic = 1;
            s = gemm(g, split_for(ld.Ppad, H), st);
        }
        if (s != PS_OK) return s;
        // dA2 = G W3 (the adjoint of A2) times SiLU'(Z2): dZ2 as bfloat16; db2 += its column sums
        w = bwg::Args{};
        w.A = f->Gb; w.lam = 1; w.lak = ldg; w.B = f->pb + ld.off_W3; w.ldb = H;
        w.M = Bi; w.N = H; w.K = ld.Ppad; w.Zs = Z2; w.ldz = H; w.Cb = f->dZb; w.ldcb = H;
        w.colsum = f->grad + ld.off_b2;
        if (!gemm_bw(w, true, bwg::kSiluGrad, 1, st, &s)) {
            GemmArgs g{};
            g.A = f->Gb; g.lam = 1; g.lak = ldg; g.B = f->pb + ld.off_W3; g.lbn = 1; g.lbk = H;
            g.M = Bi; g.N = H; g.K = ld.Ppad; g.C = f->dZ; g.ldc = H; g.Cb = f->dZb; g.ldcb = H;
            g.act = 2; g.Zs = Z2;
            s = gemm(g, 1, st);
            if (s == PS_OK) {
                k_colsum<<<dim3(blocks(H, 64), colsum_rows), 64, 0, st>>>(B, H, f->dZ, f->grad + ld.off_b2);
                launches += 1;
            }
        }
        if (s != PS_OK) return s;
        // middle layer: dW2 += dZ2^T A1, dA1 = (dZ2 W2) x SiLU'(Z1), db1 += its column sums
        w = bwg::Args{};
        w.A = f->dZb; w.lam = 1; w.lak = H; w.B = A1; w.ldb = H;
        w.M = H; w.N = H; w.K = Bi; w.C = f->grad + ld.off_W2; w.ldc = H;
        if (!gemm_bw(w, true, bwg::kAtomic, split_bw(H, H), st, &s)) {
            GemmArgs g{};
            g.A = f->dZb; g.lam = 1; g.lak = H; g.B = A1; g.lbn = 1; g.lbk = H;
            g.M = H; g.N = H; g.K = Bi; g.C = f->grad + ld.off_W2; g.ldc = H; g.atomic = 1;
            s = gemm(g, split_for(H, H), st);
        }
        if (s != PS_OK) return s;
        w = bwg::Args{};
        w.A = f->dZb; w.lam = H; w.lak = 1; w.B = f->pb + ld.off_W2; w.ldb = H;
        w.M = Bi; w.N = H; w.K = H; w.Zs = Z1; w.ldz = H; w.Cb = f->dAb; w.ldcb = H;
        w.colsum = f->grad + ld.off_b1;
        if (!gemm_bw(w, false, bwg::kSiluGrad, 1, st, &s)) {
            GemmArgs g{};
            g.A = f->dZb; g.lam = H; g.lak = 1; g.B = f->pb + ld.off_W2; g.lbn = 1; g.lbk = H;
            g.M = Bi; g.N = H; g.K = H; g.C = f->dA; g.ldc = H; g.Cb = f->dAb; g.ldcb = H;
            g.act = 2; g.Zs = Z1;
            s = gemm(g, 1, st);
            if (s == PS_OK) {
                k_colsum<<<dim3(blocks(H, 64), colsum_rows), 64, 0, st>>>(B, H, f->dA, f->grad + ld.off_b1);
                launches += 1;
            }
        }
        if (s != PS_OK) return s;
        // first layer: dW1 += dA1^T In, dIn = dA1 W1
        w = bwg::Args{};
        w.A = f->dAb; w.lam = 1; w.lak = H; w.B = In; w.ldb = kInPad;
        w.M = H; w.N = kInPad; w.K = Bi; w.C = f->grad + ld.off_W1; w.ldc = kInPad;
        if (!gemm_bw(w, true, bwg::kAtomic, split_bw(H, kInPad), st, &s)) {
            GemmArgs g{};
            g.A = f->dAb; g.lam = 1; g.lak = H; g.B = In; g.lbn = 1; g.lbk = kInPad;
            g.M = H; g.N = kInPad; g.K = Bi; g.C = f->grad + ld.off_W1; g.ldc = kInPad; g.atomic = 1;
            s = gemm(g, split_for(H, kInPad), st);
        }
        if (s != PS_OK) return s;
        w = bwg::Args{};
        w.A = f->dAb; w.lam = H; w.lak = 1; w.B = f->pb + ld.off_W1; w.ldb = kInPad;
        w.M = Bi; w.N = kInPad; w.K = H; w.C = f->dIn; w.ldc = kInPad;
        if (!gemm_bw(w, false, bwg::kStore, 1, st, &s)) {
            GemmArgs g{};
            g.A = f->dAb; g.lam = H; g.lak = 1; g.B = f->pb + ld.off_W1; g.lbn = 1; g.lbk = kInPad;
            g.M = Bi; g.N = kInPad; g.K = H; g.C = f->dIn; g.ldc = kInPad;
            s = gemm(g, 1, st);
        }
        if (s != PS_OK) return s;
        k_scatter<<<blocks(B, T), T, 0, st>>>(B, d, ld, f->dIn, f->gXn);
        std::swap(f->gX, f->gXn);
        launches += 2;  // spline backward, scatter (the GEMMs count themselves)
    }
    ps::count_launches(launches);
    return fcheck(cudaGetLastError(), "flow backward");
}

// the fused path covers hidden width 128, at most 18 bins and 8 transformed dims per layer
bool fused_ok(const FlowDesc& fd) {
    if (fd.H != kFH || 3 * fd.K + 1 > kQRows) return false;
    for (int l = 0; l < fd.L; ++l)
        if (fd.layer[l].nb > kMaxNb) return false;
    return true;
}

int ensure_gen(ps_flow f) {
    if (f->gen_X) return PS_OK;
    // events per chunk of a generate call: each chunk runs one kernel per coupling layer, so large
    // chunks spread each launch's fixed cost (weights into shared memory, TMEM allocation, the
    // partly filled last round of tiles) over more tiles
    const int64_t cap = int64_t(1) << 22;
    int s = fcheck(cudaMalloc(&f->gen_X, cap * f->fd.d * sizeof(float)), "cudaMalloc (flow sampling)");
    if (s == PS_OK) s = fcheck(cudaMalloc(&f->gen_ld, cap * sizeof(float)), "cudaMalloc (flow sampling)");
    if (s == PS_OK) s = fcheck(cudaMalloc(&f->gen_status, sizeof(unsigned long long)), "cudaMalloc (flow sampling)");
    if (s == PS_OK) s = fcheck(cudaMemset(f->gen_status, 0, sizeof(unsigned long long)), "cudaMemset");
    if (s != PS_OK) return s;
    f->gen_cap = cap;
    // the dynamic shared memory of the fused kernel exceeds the default limit
    for (auto kern : {k_layer_fused<false, 16>, k_layer_fused<false, 0>, k_layer_fused<true, 16>,
                      k_layer_fused<true, 0>})
        if (s == PS_OK)
            s = fcheck(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(FusedSmem::total)),
                       "cudaFuncSetAttribute");
    for (auto kern : {umma::k_layer_umma<false, false>, umma::k_layer_umma<true, false>, umma::k_layer_umma<false, true>})
        if (s == PS_OK)
            s = fcheck(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            static_cast<int>(umma::Smem::total(kMaxNb))),
                       "cudaFuncSetAttribute");
    return s;
}

// all layers of the fused path on X [B][d] in place, log-determinant accumulated into ld
int fused_layers(ps_flow f, int64_t B, float* X, float* ld, bool inverse, cudaStream_t st) {
    const FlowDesc& fd = f->fd;
    if (fd.K == 16) {  // the tcgen05 form: 128 events per tile, two tiles in flight, one CTA per SM
        const int64_t tiles = (B + umma::kTile - 1) / umma::kTile;
        const unsigned grid =
            static_cast<unsigned>(std::min<int64_t>(f->sms, (tiles + umma::kInFlight - 1) / umma::kInFlight));
        for (int k = 0; k < fd.L; ++k) {
            const int l = inverse ? fd.L - 1 - k : k;
            const LayerDesc& lay = fd.layer[l];
            auto kern = inverse ? umma::k_layer_umma<true, false> : umma::k_layer_umma<false, false>;
            kern<<<grid, umma::kThreads, umma::Smem::total(lay.nb), st>>>(
                B, fd.d, X, ld, lay, f->pb + lay.off_W1, f->p + lay.off_b1, f->pb + lay.off_W2, f->p + lay.off_b2,
                f->pb + lay.off_W3, f->p + lay.off_b3, f->gen_status, f->wait_limit, f->debug_flags & 1,
                umma::TrainOut{});
        }
        ps::count_launches(fd.L);
        return fcheck(cudaGetLastError(), "k_layer_umma");
    }
    const int64_t tiles = (B + 16 * kFWarps - 1) / (16 * kFWarps);
    const unsigned grid = static_cast<unsigned>(std::min<int64_t>(f->sms, tiles));
    for (int k = 0; k < fd.L; ++k) {
        const int l = inverse ? fd.L - 1 - k : k;
        const LayerDesc& lay = fd.layer[l];
        auto kern = inverse ? (fd.K == 16 ? k_layer_fused<true, 16> : k_layer_fused<true, 0>)
                            : (fd.K == 16 ? k_layer_fused<false, 16> : k_layer_fused<false, 0>);
        kern<<<grid, kFWarps * 32, FusedSmem::total, st>>>(B, fd.d, fd.K, X, ld, lay, f->pb + lay.off_W1,
                                                            f->p + lay.off_b1, f->pb + lay.off_W2, f->p + lay.off_b2,
                                                            f->pb + lay.off_W3, f->p + lay.off_b3);
    }
    ps::count_launches(fd.L);
    return fcheck(cudaGetLastError(), "k_layer_fused");
}

// padded device layout <-> logical layout (per layer W1[H][na], b1[H], W2[H][H], b2[H], W3[P][H], b3[P])
int64_t logical_size(const FlowDesc& fd) {
    int64_t n = 0;
    for (int l = 0; l < fd.L; ++l) {
        const LayerDesc& ld = fd.layer[l];
        n += static_cast<int64_t>(fd.H) * ld.na + fd.H + static_cast<int64_t>(fd.H) * fd.H + fd.H +
             static_cast<int64_t>(ld.P) * fd.H + ld.P;
    }
    return n;
}

void to_logical(const FlowDesc& fd, const std::vector<float>& dev, float* out) {
    int64_t o = 0;
    for (int l = 0; l < fd.L; ++l) {
        const LayerDesc& ld = fd.layer[l];
        const int H = fd.H;
        for (int h = 0; h < H; ++h)
            for (int i = 0; i < ld.na; ++i) out[o++] = dev[ld.off_W1 + h * kInPad + i];
        for (int h = 0; h < H; ++h) out[o++] = dev[ld.off_b1 + h];
        for (int h = 0; h < H * H; ++h) out[o++] = dev[ld.off_W2 + h];
        for (int h = 0; h < H; ++h) out[o++] = dev[ld.off_b2 + h];
        for (int p = 0; p < ld.P; ++p)
            for (int h = 0; h < H; ++h) out[o++] = dev[ld.off_W3 + static_cast<int64_t>(p) * H + h];
        for (int p = 0; p < ld.P; ++p) out[o++] = dev[ld.off_b3 + p];
    }
}

void from_logical(const FlowDesc& fd, const float* in, std::vector<float>& dev) {
    int64_t o = 0;
    std::fill(dev.begin(), dev.end(), 0.0f);
    for (int l = 0; l < fd.L; ++l) {
        const LayerDesc& ld = fd.layer[l];
        const int H = fd.H;
        for (int h = 0; h < H; ++h)
            for (int i = 0; i < ld.na; ++i) dev[ld.off_W1 + h * kInPad + i] = in[o++];
        for (int h = 0; h < H; ++h) dev[ld.off_b1 + h] = in[o++];
        for (int h = 0; h < H * H; ++h) dev[ld.off_W2 + h] = in[o++];
        for (int h = 0; h < H; ++h) dev[ld.off_b2 + h] = in[o++];
        for (int p = 0; p < ld.P; ++p)
            for (int h = 0; h < H; ++h) dev[ld.off_W3 + static_cast<int64_t>(p) * H + h] = in[o++];
        for (int p = 0; p < ld.P; ++p) dev[ld.off_b3 + p] = in[o++];
    }
}

}  // namespace

extern "C" {

const char* ps_flow_last_error(void) { return f_err.c_str(); }

int ps_flow_create(int dims, int n_layers, int bins, int hidden, int64_t max_batch, uint64_t init_seed, int device,
                   ps_flow* out) {
    if (!out || dims < 2 || dims > kMaxDims || n_layers < 1 || n_layers > kMaxLayers || bins < 1 ||
        bins > kMaxBins || hidden < 16 || hidden % 16 != 0 || hidden > 512 || max_batch < 1 || max_batch > (1 << 24))
        return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_create: bad arguments");
    ps_flow f = new (std::nothrow) ps_flow_s;
    if (!f) return ffail(PS_ERR_CAPACITY, "out of host memory");
    FlowDesc& fd = f->fd;
    fd.d = dims;
    fd.L = n_layers;
    fd.K = bins;
    fd.H = hidden;
    int nbits = 1;
    while ((1 << nbits) < dims) ++nbits;
    int64_t off = 0;
    for (int l = 0; l < n_layers; ++l) {
        LayerDesc& ld = fd.layer[l];
        int b = l % nbits, flip = (l / nbits) % 2;
        ld.nb = ld.na = 0;
        for (int j = 0; j < dims; ++j) {
            // up to 16 dims: bit (l mod nbits) of the index, flipped every nbits layers; above 16, three
            // interleaved groups (j mod 3 == l mod 3), so that a layer transforms at most 8 dims and
            // conditions on at most 16
            const bool transformed = dims > 16 ? (j % 3 == l % 3) : (((j >> b) & 1) != flip);
            if (transformed) ld.tb[ld.nb++] = j;
            else ld.ta[ld.na++] = j;
        }
        if (ld.nb == 0 || ld.na == 0 || ld.na > kInPad) { delete f; return ffail(PS_ERR_INVALID_ARGUMENT, "bad mask"); }
        ld.P = ld.nb * (3 * bins + 1);
        ld.Ppad = (ld.P + 15) / 16 * 16;
        f->Pmax = std::max(f->Pmax, ld.Ppad);
        ld.off_W1 = off; off += static_cast<int64_t>(hidden) * kInPad;
        ld.off_b1 = off; off += hidden;
        ld.off_W2 = off; off += static_cast<int64_t>(hidden) * hidden;
        ld.off_b2 = off; off += hidden;
        ld.off_W3 = off; off += static_cast<int64_t>(ld.Ppad) * hidden;
        ld.off_b3 = off; off += ld.Ppad;
        off = (off + 7) / 8 * 8;
    }
    f->n_params = off;
    f->device = device;
    f->max_batch = max_batch;
    // initial parameters: hidden layers uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)), zero biases;
    // last layer zero with biases giving unit knot derivatives (the identity spline)
    std::vector<float> h(off, 0.0f);
    uint64_t s = init_seed;
    auto unif = [&](float a) { return a * (2.0f * static_cast<float>((splitmix(s) >> 11) * 0x1p-53) - 1.0f); };
    const float d_id = std::log(std::expm1(1.0 - kMinD));
    for (int l = 0; l < n_layers; ++l) {
        const LayerDesc& ld = fd.layer[l];
        for (int r = 0; r < hidden; ++r)
            for (int i = 0; i < ld.na; ++i) h[ld.off_W1 + r * kInPad + i] = unif(1.0f / std::sqrt(static_cast<float>(ld.na)));
        for (int r = 0; r < hidden * hidden; ++r) h[ld.off_W2 + r] = unif(1.0f / std::sqrt(static_cast<float>(hidden)));
        for (int q = 0; q < ld.nb; ++q)
            for (int k = 0; k <= bins; ++k) h[ld.off_b3 + q * (3 * bins + 1) + 2 * bins + k] = d_id;
    }
    Guard g(device);
    int st = fcheck(cudaDeviceGetAttribute(&f->sms, cudaDevAttrMultiProcessorCount, device), "SM count");
    auto alloc = [&](void** q, size_t bytes) {
        if (st == PS_OK) st = fcheck(cudaMalloc(q, std::max<size_t>(bytes, 256)), "cudaMalloc (flow)");
    };
    const int64_t B = max_batch, H = hidden, L = n_layers;
    alloc(reinterpret_cast<void**>(&f->p), off * 4);
    alloc(reinterpret_cast<void**>(&f->grad), off * 4);
    alloc(reinterpret_cast<void**>(&f->m), off * 4);
    alloc(reinterpret_cast<void**>(&f->v), off * 4);
    alloc(reinterpret_cast<void**>(&f->pb), off * 2);
    alloc(reinterpret_cast<void**>(&f->X), (L + 1) * B * dims * 4);
    alloc(reinterpret_cast<void**>(&f->In), L * B * kInPad * 2);
    alloc(reinterpret_cast<void**>(&f->Z1), L * B * H * 4);
    alloc(reinterpret_cast<void**>(&f->Z2), L * B * H * 4);
    alloc(reinterpret_cast<void**>(&f->A1), L * B * H * 2);
    alloc(reinterpret_cast<void**>(&f->A2), L * B * H * 2);
    alloc(reinterpret_cast<void**>(&f->Praw), L * B * f->Pmax * 4);
    alloc(reinterpret_cast<void**>(&f->logdet), B * 4);
    alloc(reinterpret_cast<void**>(&f->G), B * f->Pmax * 4);
    alloc(reinterpret_cast<void**>(&f->Gb), B * f->Pmax * 2);
    alloc(reinterpret_cast<void**>(&f->dA), B * H * 4);
    alloc(reinterpret_cast<void**>(&f->dZ), B * H * 4);
    alloc(reinterpret_cast<void**>(&f->dZb), B * H * 2);
    alloc(reinterpret_cast<void**>(&f->dAb), B * H * 2);
    alloc(reinterpret_cast<void**>(&f->dIn), B * kInPad * 4);
    alloc(reinterpret_cast<void**>(&f->gX), B * dims * 4);
    alloc(reinterpret_cast<void**>(&f->gXn), B * dims * 4);
    alloc(reinterpret_cast<void**>(&f->wtot), B * 8);
    alloc(reinterpret_cast<void**>(&f->scal), 2 * 8);
    if (st == PS_OK) st = fcheck(cudaMemcpy(f->p, h.data(), off * 4, cudaMemcpyHostToDevice), "upload flow params");
    if (st == PS_OK) st = fcheck(cudaMemset(f->m, 0, off * 4), "memset");
    if (st == PS_OK) st = fcheck(cudaMemset(f->v, 0, off * 4), "memset");
    if (st == PS_OK) {
        k_to_bf16<<<blocks(off, 256), 256>>>(off, f->p, f->pb);
        st = fcheck(cudaDeviceSynchronize(), "flow init");
    }
    if (st != PS_OK) { free_flow(f); delete f; return st; }
    *out = f;
    return PS_OK;
}

int ps_flow_free(ps_flow f) {
    if (!f) return PS_OK;
    {
        Guard g(f->device);
        free_flow(f);
    }
    delete f;
    return PS_OK;
}

int ps_flow_info(ps_flow f, int* dims, int* n_layers, int* bins, int* hidden, int64_t* n_params) {
    if (!f) return ffail(PS_ERR_INVALID_ARGUMENT, "null flow");
    if (dims) *dims = f->fd.d;
    if (n_layers) *n_layers = f->fd.L;
    if (bins) *bins = f->fd.K;
    if (hidden) *hidden = f->fd.H;
    if (n_params) *n_params = logical_size(f->fd);
    return PS_OK;
}

int ps_flow_mask(ps_flow f, int layer, int* transformed, int* n_transformed) {
    if (!f || layer < 0 || layer >= f->fd.L || !transformed || !n_transformed)
        return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_mask: bad arguments");
    const LayerDesc& ld = f->fd.layer[layer];
    for (int i = 0; i < ld.nb; ++i) transformed[i] = ld.tb[i];
    *n_transformed = ld.nb;
    return PS_OK;
}

int ps_flow_get_params(ps_flow f, float* host, int64_t n) {
    if (!f || !host || n != logical_size(f->fd)) return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_get_params: bad size");
    Guard g(f->device);
    std::vector<float> dev(f->n_params);
    int st = fcheck(cudaMemcpy(dev.data(), f->p, f->n_params * 4, cudaMemcpyDeviceToHost), "download params");
    if (st != PS_OK) return st;
    to_logical(f->fd, dev, host);
    return PS_OK;
}

int ps_flow_set_params(ps_flow f, const float* host, int64_t n) {
    if (!f || !host || n != logical_size(f->fd)) return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_set_params: bad size");
    Guard g(f->device);
    std::vector<float> dev(f->n_params);
    from_logical(f->fd, host, dev);
    int st = fcheck(cudaMemcpy(f->p, dev.data(), f->n_params * 4, cudaMemcpyHostToDevice), "upload params");
    if (st != PS_OK) return st;
    k_to_bf16<<<blocks(f->n_params, 256), 256>>>(f->n_params, f->p, f->pb);
    return fcheck(cudaDeviceSynchronize(), "set params");
}

int ps_flow_sample(ps_flow f, int64_t batch, uint64_t seed, uint64_t event_offset, double* r, int64_t ld_r,
                   double* logdet, double* z, void* stream) {
    if (!f || batch < 0 || (batch > 0 && !r) || ld_r < batch) return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_sample: bad arguments");
    Guard g(f->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int64_t c0 = 0; c0 < batch; c0 += f->max_batch) {
        int64_t B = std::min(f->max_batch, batch - c0);
        int s = forward(f, B, seed, event_offset + static_cast<uint64_t>(c0), st);
        if (s != PS_OK) return s;
        const float* XL = f->X + static_cast<int64_t>(f->fd.L) * f->max_batch * f->fd.d;
        k_store_r<<<blocks(B, 256), 256, 0, st>>>(B, f->fd.d, c0, ld_r, XL, f->X, f->logdet, r, logdet, z);
        ps::count_launches(1);
        f->batch = B;
    }
    if (batch > f->max_batch) f->batch = 0;  // intermediates of the last chunk only: no training step
    return fcheck(cudaGetLastError(), "ps_flow_sample");
}

int ps_flow_generate(ps_flow f, int64_t batch, uint64_t seed, uint64_t event_offset, double* r, int64_t ld_r,
                     double* logdet, double* z, void* stream) {
    if (!f || batch < 0 || (batch > 0 && !r) || ld_r < batch)
        return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_generate: bad arguments");
    Guard g(f->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!fused_ok(f->fd)) {  // the layer-by-layer path, chunk by chunk
        int s = ps_flow_sample(f, batch, seed, event_offset, r, ld_r, logdet, z, stream);
        f->batch = 0;
        return s;
    }
    int s = ensure_gen(f);
    if (s != PS_OK) return s;
    const int d = f->fd.d;
    for (int64_t c0 = 0; c0 < batch; c0 += f->gen_cap) {
        const int64_t B = std::min(f->gen_cap, batch - c0);
        k_init_z<<<blocks(B, 256), 256, 0, st>>>(B, d, seed, event_offset + static_cast<uint64_t>(c0), f->gen_X);
        cudaMemsetAsync(f->gen_ld, 0, B * sizeof(float), st);
        int n = 1;
        if (z) {
            k_store_cols<<<blocks(B, 256), 256, 0, st>>>(B, d, c0, ld_r, f->gen_X, z);
            ++n;
        }
        s = fused_layers(f, B, f->gen_X, f->gen_ld, false, st);
        if (s != PS_OK) return s;
        k_store_cols<<<blocks(B, 256), 256, 0, st>>>(B, d, c0, ld_r, f->gen_X, r);
        ++n;
        if (logdet) {
            k_store_ld<<<blocks(B, 256), 256, 0, st>>>(B, c0, f->gen_ld, logdet);
            ++n;
        }
        ps::count_launches(n);
    }
    return fcheck(cudaGetLastError(), "ps_flow_generate");
}

int ps_flow_inverse(ps_flow f, int64_t batch, const double* r, int64_t ld_r, double* z, double* logq,
                    void* stream) {
    if (!f || batch < 0 || (batch > 0 && (!r || !z)) || ld_r < batch)
        return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_inverse: bad arguments");
    Guard g(f->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int d = f->fd.d;
    if (fused_ok(f->fd)) {
        int s = ensure_gen(f);
        if (s != PS_OK) return s;
        for (int64_t c0 = 0; c0 < batch; c0 += f->gen_cap) {
            const int64_t B = std::min(f->gen_cap, batch - c0);
            k_load_r<<<blocks(B, 256), 256, 0, st>>>(B, d, c0, ld_r, r, f->gen_X);
            cudaMemsetAsync(f->gen_ld, 0, B * sizeof(float), st);
            s = fused_layers(f, B, f->gen_X, f->gen_ld, true, st);
            if (s != PS_OK) return s;
            k_store_cols<<<blocks(B, 256), 256, 0, st>>>(B, d, c0, ld_r, f->gen_X, z);
            int n = 2;
            if (logq) {
                k_store_ld<<<blocks(B, 256), 256, 0, st>>>(B, c0, f->gen_ld, logq);
                ++n;
            }
            ps::count_launches(n);
        }
        return fcheck(cudaGetLastError(), "ps_flow_inverse");
    }
    float* XL = f->X + static_cast<int64_t>(f->fd.L) * f->max_batch * d;
    for (int64_t c0 = 0; c0 < batch; c0 += f->max_batch) {
        int64_t B = std::min(f->max_batch, batch - c0);
        k_load_r<<<blocks(B, 256), 256, 0, st>>>(B, d, c0, ld_r, r, XL);
        int s = inverse(f, B, st);
        if (s != PS_OK) return s;
        // z = X[0]; logq from f->logdet
        k_store_r<<<blocks(B, 256), 256, 0, st>>>(B, d, c0, ld_r, f->X, f->X, f->logdet, z, logq, nullptr);
        ps::count_launches(2);
    }
    f->batch = 0;  // the stored activations are no longer those of a sampled batch
    return fcheck(cudaGetLastError(), "ps_flow_inverse");
}

int ps_flow_weights(ps_flow f, int64_t batch, const double* w_map, const double* logdet, double* w, void* stream) {
    if (!f || (batch > 0 && (!w_map || !logdet || !w))) return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_weights: bad arguments");
    Guard g(f->device);
    if (batch > 0) {
        k_combine<<<blocks(batch, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(batch, w_map, logdet, w);
        ps::count_launches(1);
    }
    return fcheck(cudaGetLastError(), "ps_flow_weights");
}

static int prepare_grads(ps_flow f, const double* w_map, cudaStream_t st) {
    if (f->batch <= 0) return ffail(PS_ERR_INVALID_ARGUMENT, "no sampled batch to train on (sample <= max_batch first)");
    const int64_t B = f->batch;
    cudaMemsetAsync(f->scal, 0, 2 * sizeof(double), st);
    k_weights<<<blocks(B, 256), 256, 0, st>>>(B, w_map, f->logdet, f->wtot, f->scal);
    ps::count_launches(1);
    return backward(f, B, st);
}

int ps_flow_gradients(ps_flow f, const double* w_map, float* host, int64_t n, double* loss, void* stream) {
    if (!f || !w_map || !host || n != logical_size(f->fd)) return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_gradients: bad arguments");
    Guard g(f->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int s = prepare_grads(f, w_map, st);
    if (s != PS_OK) return s;
    std::vector<float> dev(f->n_params);
    double sc[2];
    s = fcheck(cudaMemcpyAsync(dev.data(), f->grad, f->n_params * 4, cudaMemcpyDeviceToHost, st), "download grads");
    if (s == PS_OK) s = fcheck(cudaMemcpyAsync(sc, f->scal, sizeof sc, cudaMemcpyDeviceToHost, st), "download loss");
    if (s == PS_OK) s = fcheck(cudaStreamSynchronize(st), "sync");
    if (s != PS_OK) return s;
    to_logical(f->fd, dev, host);
    if (loss) *loss = sc[1];
    return PS_OK;
}

int ps_flow_train_step(ps_flow f, const double* w_map, double lr, void* stream) {
    if (!f || !w_map || !(lr > 0.0)) return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_train_step: bad arguments");
    Guard g(f->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int s = prepare_grads(f, w_map, st);
    if (s != PS_OK) return s;
    f->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.0f - std::pow(b1, static_cast<float>(f->step)), c2 = 1.0f - std::pow(b2, static_cast<float>(f->step));
    k_adam<<<blocks(f->n_params, 256), 256, 0, st>>>(f->n_params, f->p, f->grad, f->m, f->v, f->pb,
                                                     static_cast<float>(lr), b1, b2, 1e-8f, c1, c2);
    ps::count_launches(1);
    return fcheck(cudaGetLastError(), "ps_flow_train_step");
}

int ps_flow_status(ps_flow f, int64_t* timeouts) {
    if (!f || !timeouts) return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_status: bad arguments");
    *timeouts = 0;
    if (!f->gen_status) return PS_OK;
    Guard g(f->device);
    unsigned long long v = 0;
    int s = fcheck(cudaDeviceSynchronize(), "ps_flow_status");
    if (s == PS_OK) s = fcheck(cudaMemcpy(&v, f->gen_status, sizeof v, cudaMemcpyDeviceToHost), "ps_flow_status");
    if (s == PS_OK) s = fcheck(cudaMemset(f->gen_status, 0, sizeof v), "ps_flow_status");
    if (s != PS_OK) return s;
    *timeouts = static_cast<int64_t>(v);
    return PS_OK;
}

int ps_flow_set_wait_limit(ps_flow f, int polls) {
    if (!f) return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_set_wait_limit: null flow");
    f->wait_limit = polls > 0 ? polls : umma::kWaitPolls;
    return PS_OK;
}

int ps_flow_set_debug(ps_flow f, int flags) {
    if (!f || flags < 0 || flags > 3) return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_set_debug: bad arguments");
    f->debug_flags = flags;
    return PS_OK;
}

int ps_flow_loss(ps_flow f, double* loss, double* sum_w, void* stream) {
    if (!f || !loss) return ffail(PS_ERR_INVALID_ARGUMENT, "ps_flow_loss: bad arguments");
    Guard g(f->device);
    double sc[2];
    int s = fcheck(cudaMemcpyAsync(sc, f->scal, sizeof sc, cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)), "loss");
    if (s == PS_OK) s = fcheck(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "sync");
    if (s != PS_OK) return s;
    *loss = sc[1];
    if (sum_w) *sum_w = sc[0];
    return PS_OK;
}

}  // extern "C"
