// launch_params.h -- the launch description shared by the host runtime (graph.cpp), the
// interpreter kernels (kernels.cu) and the kernels compiled at run time (jit.cpp): plain
// structures of fixed-width integers and pointers, so that NVRTC compiles it as well.
#pragma once

#include <cstdint>

namespace ps {

constexpr int kMaxChannels = 32;
constexpr int kOpOutput = 1000;  // pseudo-op closing each channel's byte-code
// The shared-memory region of a CTA's staged grid starts with a table of cos and sin of 2 pi k /
// kTrigN (k < kTrigN, as (cos, sin) pairs), the FP64 kernels' azimuth table; the VEGAS grid
// follows it.
constexpr int kTrigN = 256;
constexpr int kTrigDoubles = 2 * kTrigN;

// ---------------------------------------------------------------- launch description
struct ChannelLaunch {
    int32_t code_off, code_len;    // ints in the code buffer
    int32_t imm_off, imm_len;      // doubles in the immediates buffer
    int32_t grid_off;              // doubles in the grid buffer
    int32_t vdims, vbins;
    int32_t n_slots;
    int32_t n_random;
    int32_t hist_off;              // doubles in the histogram buffer
    int32_t channel;               // the program's channel index (selects a compiled channel's code)
    int64_t n_events;
    int64_t col_off;               // first output column
    int64_t tile_begin;            // first global tile index
    int64_t ev_offset;             // event id of the channel's first event
};

struct LaunchParams {
    int32_t n_ch;
    int32_t block;                 // threads per CTA = events per tile
    int32_t smem_code_ints, smem_imm, smem_grid, smem_slots;  // per-CTA staging sizes
    int64_t n_tiles;
    const int32_t* code;
    const double* imm;
    const double* grid;
    // inputs
    const double* r;               // explicit-input mode (SoA), or nullptr for Philox
    int64_t ld_r;
    uint64_t seed;
    // outputs: f64 in FP64 programs; momenta, x1, x2 and alpha are f32 in mixed programs
    void* mom;
    void* x1;
    void* x2;
    double* w;
    void* alpha;
    int64_t ld;
    int32_t mixed;
    // scratch and program state
    double* tile_partials;         // [n_tiles][4]
    double* hist;                  // VEGAS histograms (program-owned), or nullptr
    unsigned long long* status;    // [4]
    const int32_t* stats_mode;     // device flag: nonzero adds each launch's sums into the statistics
    ChannelLaunch ch[kMaxChannels];
};

}  // namespace ps
