// jit.cpp -- compiled programs: every channel's instruction list (the paper's compute graph,
// Sec. 3.1) written out as straight-line CUDA and compiled at run time with NVRTC for sm_103a.
//
// The generated kernel runs the same op implementations as the interpreter (map_device.cuh),
// instantiated on a register frame: the slot file lives in registers, the byte-code's slot
// indices and immediates become compile-time constants, and the compiler can fold constant
// sub-expressions (M^2, M Gamma, 1/(M Gamma) ...), fuse multiply-adds across op boundaries and
// cancel the float<->double round trips of the mixed form.  The tile loop, inputs, outputs and
// per-tile sums are the interpreter's (map_tiles).  Modules are cached per device and source.
//
// A program of many channels is written as one relocatable unit per channel and a kernel unit
// that dispatches on the channel; NVRTC compiles the units concurrently on host threads (each
// thread its own NVRTC program) and nvJitLink links them into one kernel.  A requested number of
// CTAs per SM becomes the kernel's launch bounds and the channel units' register cap.
//
// The driver API (module load, launch, occupancy) is opened with dlopen at first use, so the
// library also loads on machines without a GPU driver.
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvJitLink.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <cinttypes>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ps_internal.h"

namespace ps {
namespace {

// Header texts for NVRTC, embedded at build time: kJitHeaderNames[], kJitHeaderTexts[], kJitHeaderCount.
#include "jit_sources.inc"

// Stand-ins for the standard headers that the device headers include; NVRTC has the CUDA math
// functions built in.
const char* kStdInt =
    "#pragma once\n"
    "typedef signed char int8_t; typedef short int16_t; typedef int int32_t; typedef long long int64_t;\n"
    "typedef unsigned char uint8_t; typedef unsigned short uint16_t; typedef unsigned int uint32_t;\n"
    "typedef unsigned long long uint64_t;\n"
    "namespace std { using ::int8_t; using ::int16_t; using ::int32_t; using ::int64_t; using ::uint8_t;\n"
    "using ::uint16_t; using ::uint32_t; using ::uint64_t; }\n";
const char* kStdIntC =
    "#pragma once\n"
    "typedef signed char int8_t; typedef short int16_t; typedef int int32_t; typedef long long int64_t;\n"
    "typedef unsigned char uint8_t; typedef unsigned short uint16_t; typedef unsigned int uint32_t;\n"
    "typedef unsigned long long uint64_t;\n";
const char* kStdDef = "#pragma once\n";
const char* kCmath = "#pragma once\n";

std::string hexlit(double v) {
    char b[64];
    std::snprintf(b, sizeof b, "%a", v);
    return b;
}

std::string ints(const int32_t* p, int n) {
    std::string s;
    for (int i = 0; i < n; ++i) {
        if (i) s += ", ";
        s += std::to_string(p[i]);
    }
    return s;
}

bool all_finite(const std::vector<double>& v) {
    for (double x : v)
        if (!(x == x) || x > 1.7e308 || x < -1.7e308) return false;
    return true;
}

// The invariants s = q^2 of a channel's SDE weights, each computed once per event: the channel
// weights of all other channels (one PS_OP_CHANNEL_WEIGHT each) share most of their momentum
// sums (81 distinct among 110 propagators in a 2->8 channel). An invariant is named by how it
// is formed (kind, p_a, the summed slots in order); the expression is the one the interpreter
// evaluates, so the values are the same bits.
struct InvariantMemo {
    std::map<std::string, std::string> names;           // formation -> variable
    std::map<std::string, std::vector<int32_t>> reads;  // formation -> slots it reads
    int next = 0;
    // an op wrote slots [o, o + 4): forget the invariants that read them
    void written(int32_t o) {
        for (auto it = reads.begin(); it != reads.end();) {
            bool hit = false;
            for (int32_t r : it->second) hit |= (r >= o && r < o + 4);
            if (hit) {
                names.erase(it->first);
                it = reads.erase(it);
            } else {
                ++it;
            }
        }
    }
};

// The SDE weight of another channel (PS_OP_CHANNEL_WEIGHT: k, p_a, q_1..q_k, (kind, mask, M,
// Gamma)...) as straight-line code: each propagator's invariant from the memo (declared in *decl
// before the op's block at its first use), the propagator arithmetic from the interpreter's
// sde_factor_s.
std::string channel_weight_source(const Compiled& C, const int32_t* a, int na, bool mixed, InvariantMemo* memo,
                                  std::string* decl) {
    auto imm = [&](int32_t arg) { return C.imm[~arg]; };
    const int k = static_cast<int>(imm(a[0]));
    const int32_t out = a[na];
    const std::string ldp = mixed ? "dev::mx::ldp(f, " : "dev::ldp(f, ";
    std::string s = "                {";
    s += mixed ? " float acc = 1.0f; int ex = 0;\n" : " double den = 1.0, P = 1.0;\n";
    for (int j = 2 + k; j + 3 < na; j += 4) {
        const int kind = static_cast<int>(imm(a[j]));
        const int mask = static_cast<int>(imm(a[j + 1]));
        const double M = imm(a[j + 2]), G = imm(a[j + 3]);
        std::string form = std::to_string(kind) + (kind == 1 ? ":" + std::to_string(a[1]) : std::string());
        std::vector<int32_t> reads;
        if (kind == 1) reads.push_back(a[1]);
        for (int i = 0; i < k; ++i)
            if ((mask >> i) & 1) {
                form += "," + std::to_string(a[2 + i]);
                reads.push_back(a[2 + i]);
            }
        auto it = memo->names.find(form);
        std::string var;
        if (it != memo->names.end()) {
            var = it->second;
        } else {
            var = "cw" + std::to_string(memo->next++);
            std::string q = kind == 1 ? ldp + std::to_string(a[1]) + ")"
                                      : (mixed ? "dev::mx::F4{0.0f, 0.0f, 0.0f, 0.0f}" : "dev::P4{0.0, 0.0, 0.0, 0.0}");
            for (int i = 0; i < k; ++i) {
                if (!((mask >> i) & 1)) continue;
                const std::string fn = mixed ? (kind == 1 ? "dev::mx::f4_sub(" : "dev::mx::f4_add(")
                                             : (kind == 1 ? "dev::p4_sub(" : "dev::p4_add(");
                q = fn + q + ", " + ldp + std::to_string(a[2 + i]) + "))";
            }
            *decl += mixed ? "                const float " + var + " = dev::mx::sde_sq(" + q + ");\n"
                           : "                const double " + var + " = dev::p4_sq(" + q + ");\n";
            memo->names[form] = var;
            memo->reads[form] = reads;
        }
        if (mixed)
            s += "                  dev::mx::sde_factor_s(acc, ex, " + var + ", " + std::to_string(kind) +
                 ", static_cast<float>(" + hexlit(M) + "), static_cast<float>(" + hexlit(G) + "));\n";
        else
            s += "                  dev::sde_factor_s(den, P, " + var + ", " + std::to_string(kind) + ", " + hexlit(M) +
                 ", " + hexlit(G) + ");\n";
    }
    s += mixed ? "                  dev::st(f, " + std::to_string(out) + ", dev::mx::sde_weight(acc, ex)); }\n"
               : "                  dev::st(f, " + std::to_string(out) + ", P / den); }\n";
    return s;
}

}  // namespace

namespace {
// The immediates of channel c as constexpr functions of their index: a constant index folds to a
// literal (an array would be a device variable, whose loads the compiler cannot fold).
std::string imm_source(const Compiled& C, size_t c) {
    std::string s = "struct I" + std::to_string(c) + " {\n    static __forceinline__ constexpr double v(int i) {\n        switch (i) {\n";
    for (size_t i = 0; i < C.imm.size(); ++i)
        s += "            case " + std::to_string(i) + ": return " + hexlit(C.imm[i]) + ";\n";
    s += "            default: return 0.0;\n        }\n    }\n"
         "    static __forceinline__ constexpr float f(int i) { return static_cast<float>(v(i)); }\n};\n";
    return s;
}

// One channel's event: its instruction list on a register frame, from the inputs to the stores.
// Names in scope: lp, C, ev, local, active, s_grid, cut.
std::string channel_body(const Compiled& C, size_t c, bool mixed) {
    const std::string cs = std::to_string(c);
    std::string s;
    s += std::string("                const dev::") + (mixed ? "MixRegFrame<" : "RegFrame<") +
         std::to_string(std::max(C.n_slots, 1)) + ", I" + cs + "> f{};\n";
    s += "                dev::load_inputs<kMix>(f, lp, " + cs + ", " + std::to_string(C.n_random) + ", ev, local, active);\n";
    size_t pc = 0;
    InvariantMemo memo;
    while (pc < C.code.size() && C.code[pc] != kOpOutput) {
        const int op = C.code[pc], na = C.code[pc + 1], no = C.code[pc + 2];
        const int32_t* a = C.code.data() + pc + 3;
        if (op == PS_OP_CHANNEL_WEIGHT) {  // unrolled here: counts, kinds and masks are known now
            std::string decl;
            const std::string body = channel_weight_source(C, a, na, mixed, &memo, &decl);
            s += decl + body;
            for (int i = 0; i < no; ++i) memo.written(a[na + i]);
            pc += 3 + na + no;
            continue;
        }
        for (int i = 0; i < no; ++i) memo.written(a[na + i]);
        s += "                {";
        s += na ? " constexpr int32_t a[] = {" + ints(a, na) + "};" : " const int32_t* a = nullptr;";
        s += no ? " constexpr int32_t o[] = {" + ints(a + na, no) + "};" : " const int32_t* o = nullptr;";
        if (mixed)
            s += " dev::exec_op_mixed(" + std::to_string(op) + ", a, o, " + std::to_string(na) + ", " +
                 std::to_string(no) + ", f, reinterpret_cast<const float*>(s_grid), C.vbins, cut, active); }\n";
        else
            s += " dev::exec_op(" + std::to_string(op) + ", a, o, " + std::to_string(na) + ", " + std::to_string(no) +
                 ", f, s_grid, C.vbins, cut, active); }\n";
        pc += 3 + na + no;
    }
    const int n_out = pc + 1 < C.code.size() ? C.code[pc + 1] : 0;
    s += "                constexpr int32_t od[] = {" +
         (n_out ? ints(C.code.data() + pc + 3, 2 * n_out) : std::string("0, 0")) + "};\n";
    s += "                return dev::store_outputs<kMix>(f, od, " + std::to_string(n_out) + ", lp, C, local, active);\n";
    return s;
}

const char* kChanParams =
    "(const ps::LaunchParams& lp, const ps::ChannelLaunch& C, int64_t ev, int64_t local, bool active, "
    "double* s_grid, unsigned long long* cut)";

std::string kernel_source(int block, int min_blocks) {
    const std::string bounds =
        std::to_string(block) + (min_blocks > 0 ? ", " + std::to_string(min_blocks) : std::string());
    return "extern \"C\" __global__ void __launch_bounds__(" + bounds +
           ") ps_jit_map(const __grid_constant__ ps::LaunchParams lp) {\n"
           "    extern __shared__ __align__(16) double smem[];\n"
           "    ps::dev::CompiledPolicy<psjit::kMix, psjit::Events> pol{lp, smem};\n"
           "    ps::dev::map_tiles(lp, pol, smem + lp.smem_grid);\n"
           "}\n";
}

std::string prologue(bool mixed) {
    return std::string("#include \"map_device.cuh\"\n\nnamespace psjit {\nusing namespace ps;\n") +
           (mixed ? "constexpr bool kMix = true;\n" : "constexpr bool kMix = false;\n");
}
}  // namespace

// The CUDA source of a compiled program (all channels, one precision, one block size).
std::string jit_source(const std::vector<Compiled>& ch, int block, int min_blocks, bool mixed) {
    std::string s = prologue(mixed);
    for (size_t c = 0; c < ch.size(); ++c) s += imm_source(ch[c], c);
    s += "struct Events {\n"
         "    static __device__ __forceinline__ double run(int c, const LaunchParams& lp, const ChannelLaunch& C,\n"
         "                                                 int64_t ev, int64_t local, bool active, double* s_grid,\n"
         "                                                 unsigned long long* cut) {\n"
         "        switch (C.channel) {\n";
    for (size_t c = 0; c < ch.size(); ++c) {
        s += "            case " + std::to_string(c) + ": {\n" + channel_body(ch[c], c, mixed) + "            }\n";
    }
    s += "        }\n        return 0.0;\n    }\n};\n}  // namespace psjit\n\n";
    return s + kernel_source(block, min_blocks);
}

// The split form of a large program: one unit per channel, each defining the channel's event as
// an external device function, and a kernel unit that dispatches on the channel. The units are
// compiled separately (in parallel) as relocatable code and linked into one kernel.
std::vector<std::string> jit_sources_split(const std::vector<Compiled>& ch, int block, int min_blocks, bool mixed) {
    std::vector<std::string> units;
    std::string k = prologue(mixed) + "}  // namespace psjit\n";
    for (size_t c = 0; c < ch.size(); ++c)
        k += "extern \"C\" __device__ double psjit_channel_" + std::to_string(c) + kChanParams + ";\n";
    k += "namespace psjit {\nstruct Events {\n"
         "    static __device__ __forceinline__ double run(int c, const LaunchParams& lp, const ChannelLaunch& C,\n"
         "                                                 int64_t ev, int64_t local, bool active, double* s_grid,\n"
         "                                                 unsigned long long* cut) {\n"
         "        switch (C.channel) {\n";
    for (size_t c = 0; c < ch.size(); ++c)
        k += "            case " + std::to_string(c) + ": return psjit_channel_" + std::to_string(c) +
             "(lp, C, ev, local, active, s_grid, cut);\n";
    k += "        }\n        return 0.0;\n    }\n};\n}  // namespace psjit\n\n" + kernel_source(block, min_blocks);
    units.push_back(k);
    for (size_t c = 0; c < ch.size(); ++c) {
        std::string u = prologue(mixed) + imm_source(ch[c], c) + "}  // namespace psjit\n\n";
        u += "extern \"C\" __device__ double psjit_channel_" + std::to_string(c) + kChanParams + " {\n"
             "    using namespace ps;\n    using namespace psjit;\n    {\n" + channel_body(ch[c], c, mixed) + "    }\n}\n";
        units.push_back(u);
    }
    return units;
}

// NVRTC: source -> cubin for sm_103a (host only, no device needed).
int jit_compile(const std::string& src, std::vector<char>* cubin, std::string* log, bool relocatable, int max_regs) {
    std::vector<const char*> names, texts;
    for (int i = 0; i < kJitHeaderCount; ++i) {
        names.push_back(kJitHeaderNames[i]);
        texts.push_back(kJitHeaderTexts[i]);
    }
    const char* extra_names[] = {"cstdint", "stdint.h", "stddef.h", "cmath"};
    const char* extra_texts[] = {kStdInt, kStdIntC, kStdDef, kCmath};
    for (int i = 0; i < 4; ++i) {
        names.push_back(extra_names[i]);
        texts.push_back(extra_texts[i]);
    }
    nvrtcProgram prog;
    nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), "ps_jit.cu", static_cast<int>(names.size()), texts.data(),
                                       names.data());
    if (r != NVRTC_SUCCESS) {
        *log = std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r);
        return PS_ERR_CUDA;
    }
    std::vector<const char*> opts = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device"};
    if (relocatable) opts.push_back("--relocatable-device-code=true");
    const std::string regs = "--maxrregcount=" + std::to_string(max_regs);
    if (max_regs > 0) opts.push_back(regs.c_str());
    if (std::getenv("PS_JIT_PTXAS_VERBOSE")) opts.push_back("--ptxas-options=-v");  // register and spill report in the log
    r = nvrtcCompileProgram(prog, static_cast<int>(opts.size()), opts.data());
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string lg(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &lg[0]);
    *log = lg;
    if (r != NVRTC_SUCCESS) {
        nvrtcDestroyProgram(&prog);
        return PS_ERR_GRAPH;
    }
    size_t cn = 0;
    nvrtcGetCUBINSize(prog, &cn);
    cubin->resize(cn);
    nvrtcGetCUBIN(prog, cubin->data());
    nvrtcDestroyProgram(&prog);
    return PS_OK;
}

namespace {
void dump_source(const std::string& src) {
    if (const char* dump = std::getenv("PS_JIT_DUMP")) {  // diagnostic: the generated source
        if (FILE* fp = std::fopen(dump, "w")) {
            std::fputs(src.c_str(), fp);
            std::fclose(fp);
        }
    }
}

std::mutex g_unit_mu;
std::map<std::string, std::vector<char>> g_units;  // channel unit source -> relocatable cubin

bool split_program(size_t n_ch) {
    if (const char* e = std::getenv("PS_JIT_SPLIT")) return e[0] == '1';  // diagnostic override
    return n_ch > static_cast<size_t>(kJitInlineChannels);
}

// nvJitLink: relocatable cubins -> one executable cubin for sm_103a (host only).
int link_cubins(const std::vector<std::vector<char>>& bins, std::vector<char>* cubin, std::string* log) {
    nvJitLinkHandle h;
    const bool verbose = std::getenv("PS_JIT_PTXAS_VERBOSE") != nullptr;  // the linker's register report
    const char* opts[] = {"-arch=sm_103a", "-verbose"};
    if (nvJitLinkCreate(&h, verbose ? 2 : 1, opts) != NVJITLINK_SUCCESS) {
        *log += "nvJitLinkCreate failed\n";
        return PS_ERR_CUDA;
    }
    nvJitLinkResult r = NVJITLINK_SUCCESS;
    for (size_t i = 0; i < bins.size() && r == NVJITLINK_SUCCESS; ++i) {
        const std::string name = "ps_jit_unit_" + std::to_string(i);
        r = nvJitLinkAddData(h, NVJITLINK_INPUT_CUBIN, bins[i].data(), bins[i].size(), name.c_str());
    }
    if (r == NVJITLINK_SUCCESS) r = nvJitLinkComplete(h);
    if (r != NVJITLINK_SUCCESS) {
        size_t n = 0;
        nvJitLinkGetErrorLogSize(h, &n);
        std::string lg(n, '\0');
        if (n) nvJitLinkGetErrorLog(h, &lg[0]);
        *log += "nvJitLink: " + lg;
        nvJitLinkDestroy(&h);
        return PS_ERR_GRAPH;
    }
    size_t n = 0;
    if (verbose && nvJitLinkGetInfoLogSize(h, &n) == NVJITLINK_SUCCESS && n > 1) {
        std::string lg(n, '\0');
        nvJitLinkGetInfoLog(h, &lg[0]);
        *log += lg;
    }
    nvJitLinkGetLinkedCubinSize(h, &n);
    cubin->resize(n);
    nvJitLinkGetLinkedCubin(h, cubin->data());
    nvJitLinkDestroy(&h);
    return PS_OK;
}

// The source (or the split units joined) that identifies a compiled program in the cache.
struct Plan {
    bool split = false;
    int max_regs = 0;  // the channel units' register cap (split form; 0 = none)
    std::vector<std::string> units;
    std::string key;
};

// The register cap under which min_blocks CTAs of `block` threads fit on an SM (65536 registers,
// allocated in steps of 8 per thread), or 0 for no cap.
int register_cap(int block, int min_blocks) {
    if (min_blocks <= 0) return 0;
    const int regs = (65536 / (block * min_blocks)) & ~7;
    return std::max(32, std::min(255, regs));
}

Plan make_plan(const std::vector<Compiled>& ch, int block, int min_blocks, bool mixed) {
    Plan p;
    p.split = split_program(ch.size());
    if (p.split) {
        p.max_regs = register_cap(block, min_blocks);
        p.units = jit_sources_split(ch, block, min_blocks, mixed);
        for (const std::string& u : p.units) p.key += u + "\n// ---- unit\n";
        p.key += "// maxrregcount " + std::to_string(p.max_regs) + "\n";
    } else {
        p.units = {jit_source(ch, block, min_blocks, mixed)};
        p.key = p.units[0];
    }
    return p;
}

std::string unit_key(const Plan& p, size_t i) { return p.units[i] + "// maxrregcount " + std::to_string(p.max_regs); }

int build_plan(const Plan& p, std::vector<char>* cubin, std::string* log) {
    dump_source(p.key);
    if (!p.split) return jit_compile(p.units[0], cubin, log, false, 0);
    // the units are independent NVRTC programs: compile them on a pool of host threads; a unit
    // compiled before (the same channel in a program of another block size) is taken from the cache
    const size_t n = p.units.size();
    std::vector<std::vector<char>> bins(n);
    std::vector<std::string> logs(n);
    std::vector<int> sts(n, PS_OK);
    std::vector<char> cached(n, 0);
    {
        std::lock_guard<std::mutex> lock(g_unit_mu);
        for (size_t i = 0; i < n; ++i) {
            auto it = g_units.find(unit_key(p, i));
            if (it != g_units.end()) {
                bins[i] = it->second;
                cached[i] = 1;
            }
        }
    }
    std::atomic<size_t> next{0};
    auto worker = [&] {
        for (size_t i = next++; i < n; i = next++)
            if (!cached[i]) sts[i] = jit_compile(p.units[i], &bins[i], &logs[i], true, i > 0 ? p.max_regs : 0);
    };
    const size_t hw = std::max(1u, std::thread::hardware_concurrency());
    std::vector<std::thread> pool;
    for (size_t t = 1; t < std::min(n, hw); ++t) {
        try {
            pool.emplace_back(worker);
        } catch (...) {  // no more threads: the ones started (and this one) share the rest
            break;
        }
    }
    worker();
    for (std::thread& t : pool) t.join();
    int st = PS_OK;
    for (size_t i = 0; i < n; ++i) {
        *log += logs[i];
        if (sts[i] != PS_OK && st == PS_OK) st = sts[i];
    }
    if (st != PS_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_unit_mu);
        for (size_t i = 1; i < n; ++i)  // the channel units (the kernel unit depends on the block size)
            if (!cached[i]) g_units.emplace(unit_key(p, i), bins[i]);
    }
    return link_cubins(bins, cubin, log);
}
}  // namespace

int jit_build(const std::vector<Compiled>& ch, int block, int min_blocks, bool mixed, std::vector<char>* cubin,
              std::string* log) {
    return build_plan(make_plan(ch, block, min_blocks, mixed), cubin, log);
}

namespace {
// ---------------------------------------------------------------- driver API, opened at first use
typedef int CUresult_t;
typedef void* CUmodule_t;
typedef void* CUfunction_t;
struct Driver {
    bool ok = false;
    std::string why;
    CUresult_t (*moduleLoadData)(CUmodule_t*, const void*) = nullptr;
    CUresult_t (*moduleGetFunction)(CUfunction_t*, CUmodule_t, const char*) = nullptr;
    CUresult_t (*launchKernel)(CUfunction_t, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                               void*, void**, void**) = nullptr;
    CUresult_t (*occupancy)(int*, CUfunction_t, int, size_t) = nullptr;
    // kernel nodes of a captured graph: the runtime cannot read back a node whose kernel came
    // from a module loaded through the driver, so the executor reads and updates those here
    CUresult_t (*nodeGetParams)(void*, CUDA_KERNEL_NODE_PARAMS*) = nullptr;
    CUresult_t (*execNodeSetParams)(void*, void*, const CUDA_KERNEL_NODE_PARAMS*) = nullptr;
};

Driver& driver() {
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        void* h = dlopen("libcuda.so.1", RTLD_NOW | RTLD_LOCAL);
        if (!h) h = dlopen("libcuda.so", RTLD_NOW | RTLD_LOCAL);
        if (!h) {
            d.why = "the CUDA driver library could not be opened";
            return;
        }
        d.moduleLoadData = reinterpret_cast<decltype(d.moduleLoadData)>(dlsym(h, "cuModuleLoadData"));
        d.moduleGetFunction = reinterpret_cast<decltype(d.moduleGetFunction)>(dlsym(h, "cuModuleGetFunction"));
        d.launchKernel = reinterpret_cast<decltype(d.launchKernel)>(dlsym(h, "cuLaunchKernel"));
        d.occupancy = reinterpret_cast<decltype(d.occupancy)>(dlsym(h, "cuOccupancyMaxActiveBlocksPerMultiprocessor"));
        d.nodeGetParams = reinterpret_cast<decltype(d.nodeGetParams)>(dlsym(h, "cuGraphKernelNodeGetParams_v2"));
        d.execNodeSetParams =
            reinterpret_cast<decltype(d.execNodeSetParams)>(dlsym(h, "cuGraphExecKernelNodeSetParams_v2"));
        d.ok = d.moduleLoadData && d.moduleGetFunction && d.launchKernel && d.occupancy && d.nodeGetParams &&
               d.execNodeSetParams;
        if (!d.ok) d.why = "the CUDA driver library lacks a needed entry point";
    });
    return d;
}

std::mutex g_cache_mu;
std::map<std::pair<int, std::string>, CUfunction_t> g_cache;  // (device, source) -> kernel
}  // namespace

// Compile (or find in the cache) the program's kernel on the current device.
int jit_prepare(const std::vector<Compiled>& ch, int block, int min_blocks, bool mixed, int device, void** fn,
                std::string* err) {
    for (const Compiled& C : ch)
        if (!all_finite(C.imm)) {
            *err = "a channel has a non-finite immediate";
            return PS_ERR_GRAPH;
        }
    Driver& d = driver();
    if (!d.ok) {
        *err = d.why;
        return PS_ERR_CUDA;
    }
    const Plan plan = make_plan(ch, block, min_blocks, mixed);
    std::lock_guard<std::mutex> lock(g_cache_mu);
    auto key = std::make_pair(device, plan.key);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *fn = it->second;
        return PS_OK;
    }
    std::vector<char> cubin;
    std::string log;
    int st = build_plan(plan, &cubin, &log);
    if (st != PS_OK) {
        *err = "NVRTC: " + log;
        return st;
    }
    CUmodule_t mod = nullptr;
    CUfunction_t f = nullptr;
    if (d.moduleLoadData(&mod, cubin.data()) != 0 || d.moduleGetFunction(&f, mod, "ps_jit_map") != 0) {
        *err = "loading the compiled module failed";
        return PS_ERR_CUDA;
    }
    g_cache[key] = f;
    *fn = f;
    return PS_OK;
}

int jit_occupancy(void* fn, int block, size_t smem, int* per_sm) {
    Driver& d = driver();
    if (!d.ok || d.occupancy(per_sm, fn, block, smem) != 0) return PS_ERR_CUDA;
    return PS_OK;
}

int jit_launch(void* fn, const LaunchParams& lp, int grid, size_t smem, void* stream, std::string* err) {
    if (lp.n_tiles == 0) return PS_OK;
    Driver& d = driver();
    void* args[] = {const_cast<LaunchParams*>(&lp)};
    const int r = d.launchKernel(fn, static_cast<unsigned>(grid), 1, 1, static_cast<unsigned>(lp.block), 1, 1,
                                 static_cast<unsigned>(smem), stream, args, nullptr);
    if (r != 0) {
        *err = "compiled kernel launch failed (driver error " + std::to_string(r) + ")";
        return PS_ERR_CUDA;
    }
    count_launches(1);
    return PS_OK;
}

bool jit_node_runs(void* node, void* fn) {
    Driver& d = driver();
    if (!d.ok || !fn) return false;
    CUDA_KERNEL_NODE_PARAMS kp;
    std::memset(&kp, 0, sizeof(kp));
    return d.nodeGetParams(node, &kp) == 0 && static_cast<void*>(kp.func) == fn;
}

int jit_node_set(void* exec, void* node, void* fn, const LaunchParams& lp, int grid, size_t smem, std::string* err) {
    Driver& d = driver();
    if (!d.ok) {
        *err = d.why;
        return PS_ERR_CUDA;
    }
    CUDA_KERNEL_NODE_PARAMS kp;
    std::memset(&kp, 0, sizeof(kp));
    void* args[] = {const_cast<LaunchParams*>(&lp)};
    kp.func = static_cast<CUfunction>(fn);
    kp.gridDimX = static_cast<unsigned>(grid);
    kp.gridDimY = kp.gridDimZ = 1;
    kp.blockDimX = static_cast<unsigned>(lp.block);
    kp.blockDimY = kp.blockDimZ = 1;
    kp.sharedMemBytes = static_cast<unsigned>(smem);
    kp.kernelParams = args;  // copied by the call
    const int r = d.execNodeSetParams(exec, node, &kp);
    if (r != 0) {
        *err = "updating the compiled kernel's graph node failed (driver error " + std::to_string(r) + ")";
        return PS_ERR_CUDA;
    }
    return PS_OK;
}

}  // namespace ps
