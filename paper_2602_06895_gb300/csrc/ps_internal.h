// ps_internal.h -- structures shared by the host compiler (graph.cpp) and the
// device interpreter (kernels.cu) of the GB300 phase-space library.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "launch_params.h"
#include "ps.h"

namespace ps {

constexpr int kMaxOutMomenta = 24;
constexpr int kNoallocTiles = 131072;  // tiles of the allocation-free entry point's fixed scratch
constexpr int kMaxDevices = 64;
// VEGAS training histogram (kernels.cu): chunks per channel, threads per chunk, and the largest
// grid it takes (dimensions x bins <= kHistThreads * kHistEntries, bins <= 256)
constexpr int kHistChunks = 128;
constexpr int kHistThreads = 256;
constexpr int kHistEntries = 16;
constexpr int kHistMaxDims = 64;

// ---------------------------------------------------------------- graph IR
struct Arg {
    int kind;  // PS_ARG_VALUE / PS_ARG_IMM
    int id;
    double imm;
};

struct Instr {
    int op;
    std::vector<Arg> args;
    std::vector<int> outs;  // value ids
};

struct Graph {
    int n_random = 0;
    std::vector<int> type;  // value id -> PS_TYPE_*
    std::vector<Instr> code;
    std::vector<int> out_ids, out_roles;
    bool outputs_set = false;
};

// ---------------------------------------------------------------- compiled channel
// Byte-code: per instruction [op, n_args, n_out, args..., outs...]; an argument >= 0 is a
// slot index (momenta occupy 4 consecutive slots), < 0 encodes immediate ~arg.  The code
// ends with [kOpOutput, n, 0, (role, slot) x n].
struct Compiled {
    std::vector<int32_t> code;
    std::vector<double> imm;
    int n_slots = 0;
    int n_random = 0;
    int vegas_dims = 0;  // dims of the VEGAS op (0 if none)
    int n_momenta_out = 0;
    bool has_x1 = false, has_x2 = false, has_alpha = false;
};

int compile_graph(const Graph& g, Compiled* out, std::string* err);

// ---------------------------------------------------------------- inverse map plan
// Everything the inverse kernel needs about one channel, flattened on the host from its
// ps_channel_desc (the same layout, bounds recipe and propagators as the forward builder).
constexpr int kInvNodes = 32, kInvLegs = 10, kInvIds = 512, kInvProps = 40;
struct InvNode {
    int32_t kind, nch, leaf;
    int32_t child[kInvLegs];
    uint32_t mask;       // leaf-index bit mask of the subtree
    double mass, M, G, nu;
};
struct InvPlan {
    int32_t n, n_nodes, hadronic, lab_frame, kappa, n_sorder, n_pre, d, vdims, vbins;
    double S, sqrt_s, a, shat_M, shat_G, shat_nu, t_nu, ts_nu, mleaf;
    int32_t sorder[kInvNodes], pre[kInvNodes];
    int32_t d_shat, d_x, d_s[kInvNodes], d_ts[kInvLegs + 1], d_tt[kInvLegs + 1], d_tphi[kInvLegs + 1];
    int32_t d_dphi[kInvNodes], d_dth[kInvNodes];
    int32_t order[kInvLegs + 2], side[kInvLegs + 1];
    // s-order step i: m_min = lo_c + sum sqrt(s_id) over ids[lo_beg[i] .. off_beg[i]),
    // m_max = m_top - (off_c + sum sqrt(s_id) over ids[off_beg[i] .. lo_beg[i+1])),
    // m_top = sqrt(s_top) (sqrt_s for the root at fixed energy)
    double lo_c[kInvNodes], off_c[kInvNodes];
    int32_t top[kInvNodes], lo_beg[kInvNodes + 1], off_beg[kInvNodes + 1];
    int32_t ids[kInvIds];
    // propagators of the channel's SDE weight P(p): kind 0 s-channel (mask, M, G), 1 t-channel
    int32_t n_prop, pkind[kInvProps];
    uint32_t pmask[kInvProps];
    double pM[kInvProps], pG[kInvProps];
    InvNode node[kInvNodes];
};
int build_inverse_plan(const ps_channel_desc* d, InvPlan* plan, std::string* err);

// kernels.cu
int launch_map(const LaunchParams& lp, int grid_ctas, size_t smem_bytes, void* stream, std::string* err);
int launch_reduce(const LaunchParams& lp, double* stats_dev, void* stream, std::string* err);
int launch_copy(double* dst, const double* src, int n, void* stream, std::string* err);
// The VEGAS training histogram of a launch whose weights are stored (lp.hist non-null): partial
// sums per (channel, chunk) into part [n_ch][kHistChunks][stride], then added in a fixed order.
int launch_hist(const LaunchParams& lp, double* part, int stride, void* stream, std::string* err);
bool is_hist_kernel(const void* func);
void count_launches(int n);

// Compiled programs (jit.cpp): the CUDA source of a program, NVRTC to a cubin (host only), the
// cached kernel on the current device, its occupancy and its launch.
// min_blocks > 0: the kernel is compiled so that that many CTAs of `block` threads fit on an SM
// (launch bounds; the split form's channel units get the matching register cap).
std::string jit_source(const std::vector<Compiled>& ch, int block, int min_blocks, bool mixed);
int jit_compile(const std::string& src, std::vector<char>* cubin, std::string* log, bool relocatable, int max_regs);
// Programs of more than this many channels are compiled one unit per channel, in parallel, and
// linked: one unit of all channels compiles in time that grows faster than the channel count.
constexpr int kJitInlineChannels = 6;
std::vector<std::string> jit_sources_split(const std::vector<Compiled>& ch, int block, int min_blocks, bool mixed);
// The program's kernel as one executable cubin: a single unit, or the split units linked.
int jit_build(const std::vector<Compiled>& ch, int block, int min_blocks, bool mixed, std::vector<char>* cubin,
              std::string* log);
int jit_prepare(const std::vector<Compiled>& ch, int block, int min_blocks, bool mixed, int device, void** fn,
                std::string* err);
int jit_occupancy(void* fn, int block, size_t smem, int* per_sm);
int jit_launch(void* fn, const LaunchParams& lp, int grid, size_t smem, void* stream, std::string* err);
// Whether a captured kernel node runs the compiled kernel fn.
bool jit_node_runs(void* node, void* fn);
// Point an instantiated graph's compiled-kernel node at new launch parameters.
int jit_node_set(void* exec, void* node, void* fn, const LaunchParams& lp, int grid, size_t smem, std::string* err);
size_t smem_bytes_for(const LaunchParams& lp);
int max_ctas_per_sm(int block, size_t smem_bytes, int mixed, int* out, std::string* err);
// Device address and size of the fixed scratch of ps_generate_noalloc on `device` (which must be
// current); the first call on a device looks the address up.
int noalloc_scratch(int device, void** ptr, size_t* bytes, std::string* err);

// inverse.cu
int launch_inverse(const InvPlan& plan, int64_t batch, const double* mom, int64_t ld_m, const double* x1,
                   const double* x2, const double* grid, double* r, int64_t ld_r, double* P, void* stream,
                   std::string* err);
int launch_global_weights(int n_ch, int64_t batch, const double* J, int64_t ld_j, const double* P, int64_t ld_p,
                          const double* alpha, const double* x1, const double* x2, double pdf_a, double pdf_b,
                          const double* f, double* w, void* stream, std::string* err);

}  // namespace ps
