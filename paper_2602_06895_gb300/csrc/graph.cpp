// graph.cpp -- host side of the phase-space library: instruction graphs (the
// paper's compute-graph representation, Sec. 3.1), their compilation to the
// byte-code the device interpreter runs, the topology builder (Secs. 2.2.7,
// 2.2.8), programs, launches and VEGAS rebinning.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "ps_internal.h"

namespace ps {
unsigned long long launch_count();
void count_launches(int n);
bool is_reduce_kernel(const void* func);
}

using ps::Arg;
using ps::Compiled;
using ps::Graph;
using ps::Instr;

struct ps_graph_s {
    Graph g;
};

namespace {

thread_local std::string t_err;

int fail(int code, const std::string& msg) {
    t_err = msg;
    return code;
}

const char* op_name(int op) {
    switch (op) {
        case PS_OP_VEGAS: return "vegas";
        case PS_OP_INVARIANT_NU: return "stable_invariant_nu";
        case PS_OP_INVARIANT_BW: return "breit_wigner_invariant";
        case PS_OP_R_TO_X1X2: return "r_to_x1x2";
        case PS_OP_COM_P_IN: return "com_p_in";
        case PS_OP_T_INV_MIN_MAX: return "t_inv_min_max";
        case PS_OP_TWO_TO_TWO_COM: return "two_to_two_particle_scattering_com";
        case PS_OP_TWO_BODY_DECAY: return "two_body_decay";
        case PS_OP_TWO_BODY_DECAY_COM: return "two_body_decay_com";
        case PS_OP_BOOST_BEAM: return "boost_beam";
        case PS_OP_REDUCE_PRODUCT: return "reduce_product";
        case PS_OP_CUT_UNPHYSICAL: return "cut_unphysical";
        case PS_OP_ADD: return "add";
        case PS_OP_SUB: return "sub";
        case PS_OP_MUL: return "mul";
        case PS_OP_DIV: return "div";
        case PS_OP_SQRT: return "sqrt";
        case PS_OP_SQUARE: return "square";
        case PS_OP_MAX: return "max";
        case PS_OP_MOM_ADD: return "momentum_add";
        case PS_OP_MOM_SUB: return "momentum_sub";
        case PS_OP_PDF_POWER: return "pdf_power";
        case PS_OP_PROPAGATOR: return "propagator";
        case PS_OP_ONE_PLUS_COS2: return "one_plus_cos2";
        case PS_OP_CHANNEL_WEIGHT: return "channel_weight";
        default: return "?";
    }
}

// Argument type codes for signature checks.
enum { S = 1, P = 2, I = 4, SI = S | I };

// Checks the arguments of one instruction and returns the result types.
int signature(const Graph& g, int op, const std::vector<Arg>& a, std::vector<int>* outs, std::string* why) {
    auto type_of = [&](const Arg& x) -> int {
        if (x.kind == PS_ARG_IMM) return I;
        if (x.kind != PS_ARG_VALUE || x.id < 0 || x.id >= static_cast<int>(g.type.size())) return 0;
        return g.type[x.id] == PS_TYPE_MOMENTUM ? P : S;
    };
    auto expect = [&](const std::vector<int>& sig) -> bool {
        if (a.size() != sig.size()) {
            *why = std::string(op_name(op)) + ": expected " + std::to_string(sig.size()) + " arguments, got " +
                   std::to_string(a.size());
            return false;
        }
        for (size_t k = 0; k < sig.size(); ++k) {
            int t = type_of(a[k]);
            if (!(t & sig[k])) {
                *why = std::string(op_name(op)) + ": argument " + std::to_string(k) + " has the wrong type or an undefined id";
                return false;
            }
        }
        return true;
    };
    const int sc = PS_TYPE_SCALAR, mo = PS_TYPE_MOMENTUM;
    outs->clear();
    switch (op) {
        case PS_OP_VEGAS: {
            if (a.empty() || a.size() > 64) { *why = "vegas: 1..64 arguments"; return 0; }
            for (auto& x : a) if (type_of(x) != S) { *why = "vegas: arguments must be scalar values"; return 0; }
            outs->assign(a.size() + 1, sc);
            return 1;
        }
        case PS_OP_INVARIANT_NU:
            if (!expect({S, SI, I, SI, SI, I})) return 0;
            *outs = {sc, sc};
            return 1;
        case PS_OP_INVARIANT_BW:  // optional 6th: the immediate atan((x_min - M^2)/(M Gamma))
            if (a.size() == 6 ? !expect({S, I, I, SI, SI, I}) : !expect({S, I, I, SI, SI})) return 0;
            *outs = {sc, sc};
            return 1;
        case PS_OP_R_TO_X1X2:  // optional 4th immediate (any value): also return log x1, log x2
            if (a.size() == 4) {
                if (!expect({S, S, I, I})) return 0;
                *outs = {sc, sc, sc, sc, sc};
                return 1;
            }
            if (!expect({S, S, I})) return 0;
            *outs = {sc, sc, sc};
            return 1;
        case PS_OP_COM_P_IN:
            if (!expect({SI})) return 0;
            *outs = {mo, mo};
            return 1;
        case PS_OP_T_INV_MIN_MAX:
            if (!expect({SI, SI, SI, SI, SI})) return 0;
            *outs = {sc, sc};
            return 1;
        case PS_OP_TWO_TO_TWO_COM:
            if (!expect({S, P, P, S, SI, SI, SI, SI, SI})) return 0;
            *outs = {mo, mo, sc};
            return 1;
        case PS_OP_TWO_BODY_DECAY:
            if (!expect({S, S, SI, SI, SI, P})) return 0;
            *outs = {mo, mo, sc};
            return 1;
        case PS_OP_TWO_BODY_DECAY_COM:
            if (!expect({S, S, SI, SI, SI})) return 0;
            *outs = {mo, mo, sc};
            return 1;
        case PS_OP_BOOST_BEAM: {
            if (a.size() < 3) { *why = "boost_beam: at least one momentum and x1, x2"; return 0; }
            for (size_t k = 0; k + 2 < a.size(); ++k)
                if (type_of(a[k]) != P) { *why = "boost_beam: leading arguments must be momenta"; return 0; }
            if (!(type_of(a[a.size() - 2]) & S) || !(type_of(a[a.size() - 1]) & S)) {
                *why = "boost_beam: x1, x2 must be scalar values";
                return 0;
            }
            outs->assign(a.size() - 2, mo);
            return 1;
        }
        case PS_OP_REDUCE_PRODUCT: {
            if (a.empty()) { *why = "reduce_product: no arguments"; return 0; }
            for (auto& x : a) if (!(type_of(x) & SI)) { *why = "reduce_product: scalar arguments only"; return 0; }
            *outs = {sc};
            return 1;
        }
        case PS_OP_CUT_UNPHYSICAL: {
            if (a.size() < 3) { *why = "cut_unphysical: (w, x1, x2, momenta...)"; return 0; }
            if (type_of(a[0]) != S || !(type_of(a[1]) & SI) || !(type_of(a[2]) & SI)) {
                *why = "cut_unphysical: (w, x1, x2) must be scalars";
                return 0;
            }
            for (size_t k = 3; k < a.size(); ++k)
                if (type_of(a[k]) != P) { *why = "cut_unphysical: trailing arguments must be momenta"; return 0; }
            *outs = {sc};
            return 1;
        }
        case PS_OP_ADD: case PS_OP_SUB: case PS_OP_MUL: case PS_OP_DIV: case PS_OP_MAX:
            if (!expect({SI, SI})) return 0;
            *outs = {sc};
            return 1;
        case PS_OP_SQRT: case PS_OP_SQUARE:
            if (!expect({S})) return 0;
            *outs = {sc};
            return 1;
        case PS_OP_MOM_ADD: case PS_OP_MOM_SUB:
            if (!expect({P, P})) return 0;
            *outs = {mo};
            return 1;
        case PS_OP_PDF_POWER:  // optional 4th: log x; the pair form adds x2, log x2
            if (a.size() == 6 ? !expect({S, I, I, S, S, S})
                              : (a.size() == 4 ? !expect({S, I, I, S}) : !expect({S, I, I})))
                return 0;
            *outs = {sc};
            return 1;
        case PS_OP_PROPAGATOR:
            if (!expect({S, I, I})) return 0;
            *outs = {sc};
            return 1;
        case PS_OP_ONE_PLUS_COS2:
            if (!expect({P})) return 0;
            *outs = {sc};
            return 1;
        case PS_OP_CHANNEL_WEIGHT: {
            if (a.empty() || a[0].kind != PS_ARG_IMM) { *why = "channel_weight: first argument is the immediate k"; return 0; }
            int k = static_cast<int>(a[0].imm);
            if (k < 0 || k > 30 || a.size() < static_cast<size_t>(2 + k) || (a.size() - 2 - k) % 4 != 0) {
                *why = "channel_weight: (k, p_a, q_1..q_k, (kind, mask, M, Gamma)...)";
                return 0;
            }
            for (int j = 1; j < 2 + k; ++j)
                if (type_of(a[j]) != P) { *why = "channel_weight: momenta expected"; return 0; }
            for (size_t j = 2 + k; j < a.size(); ++j)
                if (type_of(a[j]) != I) { *why = "channel_weight: propagator table must be immediate"; return 0; }
            *outs = {sc};
            return 1;
        }
        default:
            *why = "unknown opcode " + std::to_string(op);
            return 0;
    }
}

}  // namespace

// ===================================================================== compile
namespace ps {

int compile_graph(const Graph& g, Compiled* out, std::string* err) {
    if (!g.outputs_set) { *err = "graph outputs were not set"; return PS_ERR_GRAPH; }
    const int nv = static_cast<int>(g.type.size());
    const int ni = static_cast<int>(g.code.size());
    const int kLive = 1 << 30;
    std::vector<int> last(nv, -1);
    for (int i = 0; i < ni; ++i)
        for (auto& a : g.code[i].args)
            if (a.kind == PS_ARG_VALUE) last[a.id] = i;
    for (int id : g.out_ids) last[id] = kLive;

    std::vector<int> slot(nv, -1);
    std::vector<char> used;
    auto alloc = [&](int width) {
        for (int s = 0;; ++s) {
            if (s + width > static_cast<int>(used.size())) used.resize(s + width, 0);
            bool ok = true;
            for (int k = 0; k < width; ++k) ok &= !used[s + k];
            if (ok) {
                for (int k = 0; k < width; ++k) used[s + k] = 1;
                return s;
            }
        }
    };
    auto width = [&](int id) { return g.type[id] == PS_TYPE_MOMENTUM ? 4 : 1; };
    auto release = [&](int id) { for (int k = 0; k < width(id); ++k) used[slot[id] + k] = 0; };

    for (int j = 0; j < g.n_random; ++j) slot[j] = alloc(1);  // inputs fill slots 0..n_random-1
    for (int j = 0; j < g.n_random; ++j) if (last[j] < 0) release(j);

    std::map<uint64_t, int> imm_index;  // keyed by bit pattern (keeps -0.0 and 0.0 apart)
    auto imm = [&](double v) {
        uint64_t bits;
        std::memcpy(&bits, &v, sizeof bits);
        auto it = imm_index.find(bits);
        if (it != imm_index.end()) return it->second;
        int idx = static_cast<int>(out->imm.size());
        out->imm.push_back(v);
        imm_index[bits] = idx;
        return idx;
    };

    out->code.clear();
    out->imm.clear();
    out->n_random = g.n_random;
    out->vegas_dims = 0;
    for (int i = 0; i < ni; ++i) {
        const Instr& in = g.code[i];
        if (in.op == PS_OP_VEGAS) {
            if (out->vegas_dims != 0) { *err = "at most one vegas instruction per channel"; return PS_ERR_GRAPH; }
            out->vegas_dims = static_cast<int>(in.args.size());
        }
        out->code.push_back(in.op);
        out->code.push_back(static_cast<int32_t>(in.args.size()));
        out->code.push_back(static_cast<int32_t>(in.outs.size()));
        for (auto& a : in.args) out->code.push_back(a.kind == PS_ARG_VALUE ? slot[a.id] : ~imm(a.imm));
        // In place: vegas and boost_beam read argument k before they write output k and touch no
        // other argument after that, so output k may take the slot of argument k when that
        // argument dies here (it halves the peak of the slot file at the beam boost).
        const bool in_place = in.op == PS_OP_VEGAS || in.op == PS_OP_BOOST_BEAM;
        for (size_t k = 0; k < in.outs.size(); ++k) {
            const int id = in.outs[k];
            int from = -1;
            if (in_place && k < in.args.size() && in.args[k].kind == PS_ARG_VALUE && last[in.args[k].id] == i &&
                width(in.args[k].id) == width(id)) {
                int uses = 0;
                for (auto& a : in.args) uses += (a.kind == PS_ARG_VALUE && a.id == in.args[k].id) ? 1 : 0;
                if (uses == 1) from = in.args[k].id;
            }
            if (from >= 0) {
                slot[id] = slot[from];
                last[from] = -2;  // its slot now belongs to the output
            } else {
                slot[id] = alloc(width(id));
            }
            out->code.push_back(slot[id]);
        }
        for (auto& a : in.args)
            if (a.kind == PS_ARG_VALUE && last[a.id] == i) {
                release(a.id);
                last[a.id] = -2;  // released (an id can appear twice in one instruction)
            }
        for (int id : in.outs)
            if (last[id] < 0) release(id);
    }
    out->code.push_back(kOpOutput);
    out->code.push_back(static_cast<int32_t>(g.out_ids.size()));
    out->code.push_back(0);
    out->n_momenta_out = 0;
    out->has_x1 = out->has_x2 = out->has_alpha = false;
    for (size_t k = 0; k < g.out_ids.size(); ++k) {
        out->code.push_back(g.out_roles[k]);
        out->code.push_back(slot[g.out_ids[k]]);
        if (g.out_roles[k] == PS_ROLE_MOMENTUM) ++out->n_momenta_out;
        if (g.out_roles[k] == PS_ROLE_X1) out->has_x1 = true;
        if (g.out_roles[k] == PS_ROLE_X2) out->has_x2 = true;
        if (g.out_roles[k] == PS_ROLE_ALPHA) out->has_alpha = true;
    }
    out->n_slots = static_cast<int>(used.size());
    if (out->imm.empty()) out->imm.push_back(0.0);
    return PS_OK;
}

}  // namespace ps

// ===================================================================== graph C ABI
extern "C" {

const char* ps_last_error(void) { return t_err.c_str(); }

int ps_version(void) { return 10000; }

int ps_graph_create(int n_random, ps_graph* out) {
    if (!out || n_random < 0 || n_random > 64) return fail(PS_ERR_INVALID_ARGUMENT, "ps_graph_create: bad arguments");
    ps_graph g = new (std::nothrow) ps_graph_s;
    if (!g) return fail(PS_ERR_CAPACITY, "out of host memory");
    g->g.n_random = n_random;
    g->g.type.assign(n_random, PS_TYPE_SCALAR);
    *out = g;
    return PS_OK;
}

int ps_graph_add(ps_graph g, int opcode, const ps_arg* args, int n_args, int* out_ids, int n_out) {
    if (!g || (n_args > 0 && !args) || n_args < 0 || n_out < 0 || (n_out > 0 && !out_ids))
        return fail(PS_ERR_INVALID_ARGUMENT, "ps_graph_add: bad arguments");
    if (g->g.outputs_set) return fail(PS_ERR_GRAPH, "ps_graph_add: outputs already set");
    Instr in;
    in.op = opcode;
    for (int k = 0; k < n_args; ++k) in.args.push_back({args[k].kind, args[k].id, args[k].imm});
    std::vector<int> types;
    std::string why;
    if (!signature(g->g, opcode, in.args, &types, &why)) return fail(PS_ERR_GRAPH, why);
    if (static_cast<int>(types.size()) != n_out)
        return fail(PS_ERR_GRAPH, std::string(op_name(opcode)) + ": defines " + std::to_string(types.size()) +
                                      " values, caller expects " + std::to_string(n_out));
    for (int t : types) {
        in.outs.push_back(static_cast<int>(g->g.type.size()));
        g->g.type.push_back(t);
    }
    for (int k = 0; k < n_out; ++k) out_ids[k] = in.outs[k];
    g->g.code.push_back(std::move(in));
    return PS_OK;
}

int ps_graph_set_outputs(ps_graph g, const int* ids, const int* roles, int n) {
    if (!g || !ids || !roles || n <= 0) return fail(PS_ERR_INVALID_ARGUMENT, "ps_graph_set_outputs: bad arguments");
    int n_w = 0, n_mom = 0;
    for (int k = 0; k < n; ++k) {
        if (ids[k] < 0 || ids[k] >= static_cast<int>(g->g.type.size())) return fail(PS_ERR_GRAPH, "output id undefined");
        bool mom = g->g.type[ids[k]] == PS_TYPE_MOMENTUM;
        if (roles[k] == PS_ROLE_MOMENTUM) {
            if (!mom) return fail(PS_ERR_GRAPH, "momentum role on a scalar");
            ++n_mom;
        } else if (roles[k] >= PS_ROLE_X1 && roles[k] <= PS_ROLE_ALPHA) {
            if (mom) return fail(PS_ERR_GRAPH, "scalar role on a momentum");
            if (roles[k] == PS_ROLE_WEIGHT) ++n_w;
        } else {
            return fail(PS_ERR_GRAPH, "unknown output role");
        }
    }
    if (n_w != 1) return fail(PS_ERR_GRAPH, "exactly one weight output is required");
    if (n_mom > ps::kMaxOutMomenta) return fail(PS_ERR_CAPACITY, "too many momentum outputs");
    g->g.out_ids.assign(ids, ids + n);
    g->g.out_roles.assign(roles, roles + n);
    g->g.outputs_set = true;
    return PS_OK;
}

int ps_graph_info(ps_graph g, int* n_instructions, int* n_values, int* n_random) {
    if (!g) return fail(PS_ERR_INVALID_ARGUMENT, "ps_graph_info: null graph");
    if (n_instructions) *n_instructions = static_cast<int>(g->g.code.size());
    if (n_values) *n_values = static_cast<int>(g->g.type.size());
    if (n_random) *n_random = g->g.n_random;
    return PS_OK;
}

int ps_graph_dump(ps_graph g, char* buf, size_t cap, size_t* needed) {
    if (!g) return fail(PS_ERR_INVALID_ARGUMENT, "ps_graph_dump: null graph");
    std::string s = "Inputs:\n  %0 : float[batch_size, " + std::to_string(g->g.n_random) + "]  (ids 0.." +
                    std::to_string(g->g.n_random - 1) + ")\nInstructions:\n";
    char tmp[64];
    for (auto& in : g->g.code) {
        s += "  ";
        for (size_t k = 0; k < in.outs.size(); ++k) s += (k ? ", %" : "%") + std::to_string(in.outs[k]);
        s += std::string(" = ") + op_name(in.op) + "(";
        for (size_t k = 0; k < in.args.size(); ++k) {
            if (k) s += ", ";
            if (in.args[k].kind == PS_ARG_VALUE) s += "%" + std::to_string(in.args[k].id);
            else { std::snprintf(tmp, sizeof tmp, "%.9g", in.args[k].imm); s += tmp; }
        }
        s += ")\n";
    }
    s += "Outputs:\n";
    static const char* role[] = {"momentum", "x1", "x2", "weight", "alpha"};
    for (size_t k = 0; k < g->g.out_ids.size(); ++k)
        s += "  %" + std::to_string(g->g.out_ids[k]) + " : " + role[g->g.out_roles[k]] + "\n";
    if (needed) *needed = s.size() + 1;
    if (buf && cap > 0) {
        size_t n = std::min(cap - 1, s.size());
        std::memcpy(buf, s.data(), n);
        buf[n] = 0;
    }
    return PS_OK;
}

int ps_graph_free(ps_graph g) {
    delete g;
    return PS_OK;
}

}  // extern "C"

// ===================================================================== builder
namespace {

// A mass (or a sum of masses) as a constant plus a list of graph values.
struct Sum {
    double c = 0.0;
    std::vector<int> ids;
};

class Builder {
public:
    Builder(ps_graph g) : g_(g) {}

    int emit(int op, const std::vector<ps_arg>& a, int n_out, std::vector<int>* outs = nullptr) {
        std::vector<int> o(n_out);
        int st = ps_graph_add(g_, op, a.data(), static_cast<int>(a.size()), o.data(), n_out);
        if (st != PS_OK) throw st;
        if (outs) *outs = o;
        return o.empty() ? -1 : o[0];
    }
    static ps_arg V(int id) { return ps_arg{PS_ARG_VALUE, id, 0.0}; }
    static ps_arg C(double v) { return ps_arg{PS_ARG_IMM, -1, v}; }

    // value of a Sum as an argument (emits the additions)
    ps_arg arg(const Sum& s) {
        if (s.ids.empty()) return C(s.c);
        int acc = s.ids[0];
        for (size_t k = 1; k < s.ids.size(); ++k) acc = emit(PS_OP_ADD, {V(acc), V(s.ids[k])}, 1);
        if (s.c != 0.0) acc = emit(PS_OP_ADD, {V(acc), C(s.c)}, 1);
        return V(acc);
    }
    // square of a non-negative Sum
    ps_arg square(const Sum& s) {
        if (s.ids.empty()) return C(s.c * s.c);
        ps_arg a = arg(s);
        return V(emit(PS_OP_SQUARE, {a}, 1));
    }

private:
    ps_graph g_;
};

struct Topo {
    const ps_channel_desc* d;
    std::vector<int> parent;
    int kappa = 0;
};

void leaves_of(const ps_channel_desc* d, int j, unsigned* mask) {
    const ps_node_desc& nd = d->nodes[j];
    if (nd.kind == PS_NODE_LEAF) { *mask |= 1u << nd.leaf_index; return; }
    for (int k = 0; k < nd.n_children; ++k) leaves_of(d, nd.children[k], mask);
}

void preorder(const ps_channel_desc* d, int j, std::vector<int>* out) {
    const ps_node_desc& nd = d->nodes[j];
    if (nd.kind == PS_NODE_DECAY) out->push_back(j);
    for (int k = 0; k < nd.n_children; ++k) preorder(d, nd.children[k], out);
}

int validate_desc(const ps_channel_desc* d, std::string* why) {
    if (d->n_out < 2 || d->n_out > 24) { *why = "n_out must be 2..24"; return 0; }
    if (d->n_nodes < 1 || d->n_nodes > PS_MAX_NODES) { *why = "n_nodes out of range"; return 0; }
    int leaves = 0;
    std::vector<int> seen(d->n_nodes, 0);
    for (int j = 0; j < d->n_nodes; ++j) {
        const ps_node_desc& nd = d->nodes[j];
        if (nd.kind == PS_NODE_LEAF) {
            if (nd.leaf_index < 0 || nd.leaf_index >= d->n_out) { *why = "leaf index out of range"; return 0; }
            ++leaves;
        } else if (nd.kind == PS_NODE_DECAY) {
            if (nd.n_children != 2) { *why = "decay nodes have two children"; return 0; }
        } else if (nd.kind == PS_NODE_TCHAIN) {
            if (j != 0 || nd.n_children < 2 || nd.n_children > PS_MAX_LEGS) { *why = "t-chain only at the root, 2..10 legs"; return 0; }
        } else { *why = "unknown node kind"; return 0; }
        for (int k = 0; k < nd.n_children; ++k) {
            int c = nd.children[k];
            if (c <= 0 || c >= d->n_nodes || seen[c]) { *why = "bad child id (tree required)"; return 0; }
            seen[c] = 1;
        }
    }
    if (leaves != d->n_out) { *why = "number of leaves differs from n_out"; return 0; }
    if (d->nodes[0].kind == PS_NODE_LEAF) { *why = "root must be a decay or a t-chain"; return 0; }
    if (d->vegas_dims < 0 || d->vegas_dims > 64 || (d->vegas_dims > 0 && d->vegas_bins < 1)) { *why = "bad VEGAS size"; return 0; }
    if (d->n_sorder < 0 || d->n_sorder > PS_MAX_NODES) { *why = "bad sorder"; return 0; }
    int n_decay = 0;
    for (int j = 1; j < d->n_nodes; ++j) n_decay += d->nodes[j].kind == PS_NODE_DECAY;
    if (d->n_sorder != n_decay) { *why = "sorder must list every non-root decay node once"; return 0; }
    std::vector<int> in(d->n_nodes, 0);
    for (int i = 0; i < d->n_sorder; ++i) {
        int j = d->sorder[i];
        if (j <= 0 || j >= d->n_nodes || d->nodes[j].kind != PS_NODE_DECAY || in[j]) { *why = "bad sorder entry"; return 0; }
        in[j] = 1;
    }
    if (d->integrand < 0 || d->integrand > PS_INTEGRAND_PDF_SDE) { *why = "unknown integrand"; return 0; }
    return 1;
}

// Propagators of a channel for the SDE weights: resonant s-channel nodes (leaf mask) and the
// t-channel propagators q_k = p_a - (legs 1..k), k = 1..kappa.
struct Prop {
    int kind;
    unsigned mask;
    double M, G;
};

std::vector<Prop> sde_props(const ps_channel_desc* d) {
    std::vector<Prop> out;
    for (int j = 1; j < d->n_nodes; ++j) {
        const ps_node_desc& nd = d->nodes[j];
        if (nd.kind == PS_NODE_DECAY && nd.in_sde) {
            unsigned m = 0;
            leaves_of(d, j, &m);
            out.push_back({0, m, nd.prop_mass, nd.prop_width});
        }
    }
    if (d->nodes[0].kind == PS_NODE_TCHAIN) {
        unsigned m = 0;
        for (int k = 0; k + 1 < d->nodes[0].n_children; ++k) {
            leaves_of(d, d->nodes[0].children[k], &m);
            out.push_back({1, m, d->t_prop_mass, 0.0});
        }
    }
    return out;
}

int random_dims(const ps_channel_desc* d) {
    int kappa = d->nodes[0].kind == PS_NODE_TCHAIN ? d->nodes[0].n_children - 1 : 0;
    std::vector<int> pre;
    preorder(d, 0, &pre);
    int n = (d->hadronic ? 2 : 0) + d->n_sorder + std::max(kappa - 1, 0) + 2 * kappa + 2 * static_cast<int>(pre.size());
    return n;
}

void build(const ps_channel_desc* all, int n_ch, int which, ps_graph g) {
    const ps_channel_desc* d = &all[which];
    Builder b(g);
    using B = Builder;
    const int n = d->n_out;
    const ps_node_desc* nd = d->nodes;
    std::vector<int> parent(d->n_nodes, -1);
    for (int j = 0; j < d->n_nodes; ++j)
        for (int k = 0; k < nd[j].n_children; ++k) parent[nd[j].children[k]] = j;
    const int kappa = nd[0].kind == PS_NODE_TCHAIN ? nd[0].n_children - 1 : 0;
    std::vector<int> pre;
    preorder(d, 0, &pre);

    // ---- random-dimension layout (generalising the example graph of Sec. 3.2)
    int idx = 0;
    int d_shat = -1, d_x = -1;
    std::vector<int> d_s(d->n_nodes, -1), d_ts(PS_MAX_LEGS + 1, -1), d_tphi(PS_MAX_LEGS + 1, -1),
        d_tt(PS_MAX_LEGS + 1, -1), d_dphi(d->n_nodes, -1), d_dth(d->n_nodes, -1);
    if (d->hadronic) d_shat = idx++;
    for (int i = 0; i < d->n_sorder; ++i) d_s[d->sorder[i]] = idx++;
    for (int i = 1; i < kappa; ++i) d_ts[i] = idx++;
    if (d->hadronic) d_x = idx++;
    for (int i = 1; i <= kappa; ++i) { d_tphi[i] = idx++; d_tt[i] = idx++; }
    for (int j : pre) { d_dphi[j] = idx++; d_dth[j] = idx++; }

    // ---- VEGAS on the leading dimensions
    std::vector<int> r(idx);
    for (int j = 0; j < idx; ++j) r[j] = j;
    std::vector<ps_arg> jac;
    jac.push_back(B::C(std::pow(2.0 * 3.141592653589793238462643383279502884, 4 - 3 * n)));
    if (d->vegas_dims > 0) {
        std::vector<ps_arg> a;
        for (int j = 0; j < d->vegas_dims; ++j) a.push_back(B::V(j));
        std::vector<int> o;
        b.emit(PS_OP_VEGAS, a, d->vegas_dims + 1, &o);
        for (int j = 0; j < d->vegas_dims; ++j) r[j] = o[j];
        jac.push_back(B::V(o[d->vegas_dims]));
    }

    // Breit-Wigner arguments; with an immediate x_min the lower angle atan((x_min - M^2)/(M Gamma))
    // is a constant of the channel and goes in as a sixth immediate
    auto bw_args = [&](ps_arg rr, double M, double G, ps_arg smin, ps_arg smax) {
        std::vector<ps_arg> a = {rr, B::C(M), B::C(G), smin, smax};
        if (smin.kind == PS_ARG_IMM) a.push_back(B::C(std::atan((smin.imm - M * M) / (M * G))));
        return a;
    };

    // ---- shat (Sec. 2.2.2)
    std::vector<int> sid(d->n_nodes, -1), sqrt_id(d->n_nodes, -1);
    std::vector<char> sampled(d->n_nodes, 0);
    int shat;
    if (d->hadronic) {
        double mleaf = 0.0;
        for (int j = 0; j < d->n_nodes; ++j) if (nd[j].kind == PS_NODE_LEAF) mleaf += nd[j].mass;
        std::vector<int> o;
        if (d->shat_width > 0.0)
            b.emit(PS_OP_INVARIANT_BW, bw_args(B::V(r[d_shat]), d->shat_mass, d->shat_width, B::C(mleaf * mleaf),
                                               B::C(d->s_beam)), 2, &o);
        else
            b.emit(PS_OP_INVARIANT_NU, {B::V(r[d_shat]), B::C(d->shat_mass), B::C(d->shat_nu), B::C(mleaf * mleaf),
                                        B::C(d->s_beam), B::C(d->a_shift)}, 2, &o);
        shat = o[0];
        jac.push_back(B::V(o[1]));
        sid[0] = shat;
    } else {
        shat = -1;
    }
    sampled[0] = 1;
    auto shat_arg = [&]() { return d->hadronic ? B::V(shat) : B::C(d->sqrt_s * d->sqrt_s); };
    auto sqrt_of = [&](int j) -> int {
        if (sqrt_id[j] < 0) sqrt_id[j] = b.emit(PS_OP_SQRT, {B::V(sid[j])}, 1);
        return sqrt_id[j];
    };
    int sqrt_shat = d->hadronic ? sqrt_of(0) : -1;

    // minimal mass of a node (Sec. 2.2.7 step 2)
    std::function<void(int, Sum*)> min_mass = [&](int j, Sum* s) {
        if (nd[j].kind == PS_NODE_LEAF) { s->c += nd[j].mass; return; }
        if (sampled[j]) {
            if (j == 0 && !d->hadronic) s->c += d->sqrt_s;
            else s->ids.push_back(sqrt_of(j));
            return;
        }
        for (int k = 0; k < nd[j].n_children; ++k) min_mass(nd[j].children[k], s);
    };

    // ---- s-channel invariants with recursive bounds (Sec. 2.2.7)
    std::vector<ps_arg> own_props;  // SDE propagator factors from sampled invariants
    for (int i = 0; i < d->n_sorder; ++i) {
        int j = d->sorder[i];
        Sum lo;
        min_mass(j, &lo);
        // maximal mass: walk up until a sampled node; subtract the minimal masses branching off
        Sum off;
        int cur = j, top = -1;
        for (;;) {
            int p = parent[cur];
            for (int k = 0; k < nd[p].n_children; ++k)
                if (nd[p].children[k] != cur) min_mass(nd[p].children[k], &off);
            if (sampled[p]) { top = p; break; }
            cur = p;
        }
        ps_arg top_m = (top == 0 && !d->hadronic) ? B::C(d->sqrt_s) : B::V(sqrt_of(top));
        ps_arg mhi;
        if (off.ids.empty() && off.c == 0.0) {
            mhi = top_m;
        } else if (top_m.kind == PS_ARG_IMM && off.ids.empty()) {
            mhi = B::C(top_m.imm - off.c);
        } else {
            mhi = B::V(b.emit(PS_OP_SUB, {top_m, b.arg(off)}, 1));
        }
        ps_arg lo_a = b.arg(lo);
        ps_arg smin = lo.ids.empty() ? B::C(lo.c * lo.c) : B::V(b.emit(PS_OP_SQUARE, {lo_a}, 1));
        // s_max = max(m_max, m_min)^2  (empty range collapses to s_min)
        ps_arg smax;
        if (mhi.kind == PS_ARG_IMM && lo_a.kind == PS_ARG_IMM) {
            double m = std::max(mhi.imm, lo_a.imm);
            smax = B::C(m * m);
        } else {
            int mm = b.emit(PS_OP_MAX, {mhi, lo_a}, 1);
            smax = B::V(b.emit(PS_OP_SQUARE, {B::V(mm)}, 1));
        }
        std::vector<int> o;
        if (nd[j].prop_width > 0.0)
            b.emit(PS_OP_INVARIANT_BW, bw_args(B::V(r[d_s[j]]), nd[j].prop_mass, nd[j].prop_width, smin, smax), 2, &o);
        else
            b.emit(PS_OP_INVARIANT_NU, {B::V(r[d_s[j]]), B::C(nd[j].prop_mass), B::C(nd[j].nu), smin, smax,
                                        B::C(d->a_shift)}, 2, &o);
        sid[j] = o[0];
        sampled[j] = 1;
        jac.push_back(B::V(o[1]));
        if (nd[j].in_sde)
            own_props.push_back(B::V(b.emit(PS_OP_PROPAGATOR, {B::V(o[0]), B::C(nd[j].prop_mass), B::C(nd[j].prop_width)}, 1)));
    }

    // leg masses (leaf mass or sqrt of the sampled invariant)
    auto leg_mass = [&](int j) -> ps_arg {
        if (nd[j].kind == PS_NODE_LEAF) return B::C(nd[j].mass);
        return B::V(sqrt_of(j));
    };

    // ---- t-chain invariants (Sec. 2.2.8), legs taken inwards from side A or B
    std::vector<int> order(kappa + 2, -1), side(kappa + 1, 0), sts(kappa + 1, -1);
    if (kappa > 0) {
        int left = 0, right = kappa;
        for (int i = 1; i < kappa; ++i) {
            if (d->tside[i] == 0) { order[i] = left++; side[i] = 0; }
            else { order[i] = right--; side[i] = 1; }
        }
        order[kappa] = left;
        order[kappa + 1] = right;
        int l2 = 0, r2 = kappa;
        ps_arg prev = shat_arg();
        int prev_sqrt = d->hadronic ? sqrt_shat : -1;
        for (int i = 1; i < kappa; ++i) {
            if (side[i] == 0) ++l2; else --r2;
            Sum rest;
            for (int k = l2; k <= r2; ++k) {
                int c = nd[0].children[k];
                if (nd[c].kind == PS_NODE_LEAF) rest.c += nd[c].mass;
                else rest.ids.push_back(sqrt_of(c));
            }
            ps_arg smin = b.square(rest);
            ps_arg mi = leg_mass(nd[0].children[order[i]]);
            ps_arg rootp = (prev_sqrt >= 0) ? B::V(prev_sqrt)
                                             : B::C(std::sqrt(prev.imm));  // fixed energy: sqrt(s) known
            int mx = b.emit(PS_OP_SUB, {rootp, mi}, 1);
            int mxp = b.emit(PS_OP_MAX, {B::V(mx), B::C(0.0)}, 1);
            int sq = b.emit(PS_OP_SQUARE, {B::V(mxp)}, 1);
            int smax = b.emit(PS_OP_MAX, {B::V(sq), smin}, 1);
            std::vector<int> o;
            b.emit(PS_OP_INVARIANT_NU, {B::V(r[d_ts[i]]), B::C(0.0), B::C(d->ts_nu), smin, B::V(smax),
                                        B::C(d->a_shift)}, 2, &o);
            sts[i] = o[0];
            jac.push_back(B::V(o[1]));
            prev = B::V(o[0]);
            prev_sqrt = b.emit(PS_OP_SQRT, {B::V(o[0])}, 1);
        }
    }

    // ---- x1, x2 (Sec. 2.2.2)
    int x1 = -1, x2 = -1, lx1 = -1, lx2 = -1;
    if (d->hadronic) {
        std::vector<int> o;
        const bool want_logs = d->integrand == PS_INTEGRAND_PDF_PROPS || d->integrand == PS_INTEGRAND_PDF_SDE;
        if (want_logs) {  // log x = r log tau is known: the parton densities need no logarithm
            b.emit(PS_OP_R_TO_X1X2, {B::V(r[d_x]), B::V(shat), B::C(d->s_beam), B::C(1.0)}, 5, &o);
            lx1 = o[3];
            lx2 = o[4];
        } else {
            b.emit(PS_OP_R_TO_X1X2, {B::V(r[d_x]), B::V(shat), B::C(d->s_beam)}, 3, &o);
        }
        x1 = o[0];
        x2 = o[1];
        jac.push_back(B::V(o[2]));
    }

    // ---- incoming momenta in the partonic frame
    std::vector<int> po;
    b.emit(PS_OP_COM_P_IN, {d->hadronic ? B::V(sqrt_shat) : B::C(d->sqrt_s)}, 2, &po);
    const int pa = po[0], pb = po[1];
    std::vector<int> pmom(d->n_nodes, -1);

    // ---- t-chain blocks (Sec. 2.2.4 / 2.2.8)
    std::vector<ps_arg> own_t;
    if (kappa > 0) {
        int pA = pa, pB = pb;
        ps_arg mA2 = B::C(0.0), mB2 = B::C(0.0);
        ps_arg scur = shat_arg();
        for (int i = 1; i <= kappa; ++i) {
            ps_arg m1, m2;
            int leg1 = -1, leg2 = -1;
            if (i == kappa) {
                leg1 = nd[0].children[order[kappa]];
                leg2 = nd[0].children[order[kappa + 1]];
                m1 = leg_mass(leg1);
                m2 = leg_mass(leg2);
            } else if (side[i] == 0) {
                leg1 = nd[0].children[order[i]];
                m1 = leg_mass(leg1);
                m2 = B::V(b.emit(PS_OP_SQRT, {B::V(sts[i])}, 1));
            } else {
                leg1 = nd[0].children[order[i]];
                m1 = B::V(b.emit(PS_OP_SQRT, {B::V(sts[i])}, 1));
                m2 = leg_mass(leg1);
            }
            std::vector<int> tr;
            b.emit(PS_OP_T_INV_MIN_MAX, {scur, mA2, mB2, m1, m2}, 2, &tr);
            int tlo = b.emit(PS_OP_MAX, {B::V(tr[0]), B::C(0.0)}, 1);
            int thi = b.emit(PS_OP_MAX, {B::V(tr[1]), B::V(tlo)}, 1);
            std::vector<int> tt;
            b.emit(PS_OP_INVARIANT_NU, {B::V(r[d_tt[i]]), B::C(0.0), B::C(d->t_nu), B::V(tlo), B::V(thi),
                                        B::C(d->a_shift)}, 2, &tt);
            std::vector<int> blk;
            b.emit(PS_OP_TWO_TO_TWO_COM, {B::V(r[d_tphi[i]]), B::V(pA), B::V(pB), B::V(tt[0]), m1, m2, scur, mA2, mB2},
                   3, &blk);
            jac.push_back(B::V(b.emit(PS_OP_MUL, {B::V(tt[1]), B::V(blk[2])}, 1)));
            int tneg = b.emit(PS_OP_SUB, {B::C(0.0), B::V(tt[0])}, 1);
            if (d->integrand == PS_INTEGRAND_PDF_SDE)
                own_t.push_back(B::V(b.emit(PS_OP_PROPAGATOR, {B::V(tneg), B::C(d->t_prop_mass), B::C(0.0)}, 1)));
            if (i == kappa) {
                pmom[leg1] = blk[0];
                pmom[leg2] = blk[1];
            } else if (side[i] == 0) {
                pmom[leg1] = blk[0];
                pA = b.emit(PS_OP_MOM_SUB, {B::V(pA), B::V(blk[0])}, 1);
                mA2 = B::V(tneg);
                scur = B::V(sts[i]);
            } else {
                pmom[leg1] = blk[1];
                pB = b.emit(PS_OP_MOM_SUB, {B::V(pB), B::V(blk[1])}, 1);
                mB2 = B::V(tneg);
                scur = B::V(sts[i]);
            }
        }
    }

    // ---- decays in depth-first order (Sec. 2.2.3); the root decays at rest
    for (int j : pre) {
        int c1 = nd[j].children[0], c2 = nd[j].children[1];
        ps_arg m1 = leg_mass(c1), m2 = leg_mass(c2);
        std::vector<int> o;
        if (j == 0) {
            b.emit(PS_OP_TWO_BODY_DECAY_COM, {B::V(r[d_dphi[j]]), B::V(r[d_dth[j]]), shat_arg(), m1, m2}, 3, &o);
        } else {
            b.emit(PS_OP_TWO_BODY_DECAY, {B::V(r[d_dphi[j]]), B::V(r[d_dth[j]]), B::V(sid[j]), m1, m2, B::V(pmom[j])},
                   3, &o);
        }
        pmom[c1] = o[0];
        pmom[c2] = o[1];
        jac.push_back(B::V(o[2]));
    }

    // ---- event record [p_a, p_b, p_1..p_n], boosted to the lab (boost_beam)
    std::vector<int> rec(n + 2, -1);
    rec[0] = pa;
    rec[1] = pb;
    for (int j = 0; j < d->n_nodes; ++j)
        if (nd[j].kind == PS_NODE_LEAF) rec[2 + nd[j].leaf_index] = pmom[j];
    if (d->hadronic && d->lab_frame) {
        std::vector<ps_arg> a;
        for (int id : rec) a.push_back(B::V(id));
        a.push_back(B::V(x1));
        a.push_back(B::V(x2));
        std::vector<int> o;
        b.emit(PS_OP_BOOST_BEAM, a, n + 2, &o);
        rec = o;
    }

    // ---- phase-space weight (reduce_product) and integrand
    int wps = b.emit(PS_OP_REDUCE_PRODUCT, jac, 1);
    ps_arg f = B::C(1.0);
    int alpha = -1;
    auto pdfs = [&]() -> int {
        std::vector<ps_arg> a1 = {B::V(x1), B::C(d->pdf_alpha), B::C(d->pdf_beta)}, a2 = a1;
        a2[0] = B::V(x2);
        if (lx1 >= 0) {  // the pair form: one exponential for both densities
            a1.push_back(B::V(lx1));
            a1.push_back(B::V(x2));
            a1.push_back(B::V(lx2));
            return b.emit(PS_OP_PDF_POWER, a1, 1);
        }
        int f1 = b.emit(PS_OP_PDF_POWER, a1, 1);
        int f2 = b.emit(PS_OP_PDF_POWER, a2, 1);
        return b.emit(PS_OP_MUL, {B::V(f1), B::V(f2)}, 1);
    };
    if (d->integrand == PS_INTEGRAND_ONE_PLUS_COS2) {
        f = B::V(b.emit(PS_OP_ONE_PLUS_COS2, {B::V(rec[2])}, 1));
    } else if (d->integrand == PS_INTEGRAND_PDF_PROPS) {
        ps_arg props = own_props.empty() ? B::C(1.0) : B::V(b.emit(PS_OP_REDUCE_PRODUCT, own_props, 1));
        if (d->hadronic) f = B::V(b.emit(PS_OP_MUL, {B::V(pdfs()), props}, 1));
        else f = props;
    } else if (d->integrand == PS_INTEGRAND_PDF_SDE) {
        std::vector<ps_arg> fac = own_props;
        fac.insert(fac.end(), own_t.begin(), own_t.end());
        ps_arg Pc = fac.empty() ? B::C(1.0) : B::V(b.emit(PS_OP_REDUCE_PRODUCT, fac, 1));
        ps_arg sum = Pc;
        for (int c = 0; c < n_ch; ++c) {
            if (c == which) continue;
            std::vector<Prop> pr = sde_props(&all[c]);
            std::vector<ps_arg> a;
            a.push_back(B::C(n));
            a.push_back(B::V(rec[0]));
            for (int i = 0; i < n; ++i) a.push_back(B::V(rec[2 + i]));
            for (auto& p : pr) {
                a.push_back(B::C(p.kind));
                a.push_back(B::C(static_cast<double>(p.mask)));
                a.push_back(B::C(p.M));
                a.push_back(B::C(p.G));
            }
            int Pj = b.emit(PS_OP_CHANNEL_WEIGHT, a, 1);
            if (sum.kind == PS_ARG_IMM) sum = B::V(b.emit(PS_OP_ADD, {sum, B::V(Pj)}, 1));
            else sum = B::V(b.emit(PS_OP_ADD, {sum, B::V(Pj)}, 1));
        }
        if (d->hadronic) f = B::V(b.emit(PS_OP_MUL, {B::V(pdfs()), sum}, 1));
        else f = sum;
        alpha = b.emit(PS_OP_DIV, {Pc, sum}, 1);
    }
    std::vector<ps_arg> wf = {B::V(wps), f};
    if (alpha >= 0) wf.push_back(B::V(alpha));
    int w = b.emit(PS_OP_REDUCE_PRODUCT, wf, 1);

    // ---- cut_unphysical
    std::vector<ps_arg> ca = {B::V(w), d->hadronic ? B::V(x1) : B::C(1.0), d->hadronic ? B::V(x2) : B::C(1.0)};
    for (int id : rec) ca.push_back(B::V(id));
    int wc = b.emit(PS_OP_CUT_UNPHYSICAL, ca, 1);

    std::vector<int> ids, roles;
    for (int id : rec) { ids.push_back(id); roles.push_back(PS_ROLE_MOMENTUM); }
    if (d->hadronic) {
        ids.push_back(x1); roles.push_back(PS_ROLE_X1);
        ids.push_back(x2); roles.push_back(PS_ROLE_X2);
    }
    ids.push_back(wc); roles.push_back(PS_ROLE_WEIGHT);
    if (alpha >= 0) { ids.push_back(alpha); roles.push_back(PS_ROLE_ALPHA); }
    int st = ps_graph_set_outputs(g, ids.data(), roles.data(), static_cast<int>(ids.size()));
    if (st != PS_OK) throw st;
}

}  // namespace

namespace ps {
// The inverse plan of a channel: the forward builder's dimension layout, s-order bounds recipe,
// t-chain order and SDE propagators, flattened for the inverse kernel.
int build_inverse_plan(const ps_channel_desc* d, InvPlan* plan, std::string* err) {
    std::string why;
    if (!validate_desc(d, &why)) {
        *err = "channel description: " + why;
        return PS_ERR_GRAPH;
    }
    InvPlan P{};
    const ps_node_desc* nd = d->nodes;
    std::vector<int> parent(d->n_nodes, -1);
    for (int j = 0; j < d->n_nodes; ++j)
        for (int k = 0; k < nd[j].n_children; ++k) parent[nd[j].children[k]] = j;
    P.n = d->n_out;
    P.n_nodes = d->n_nodes;
    P.hadronic = d->hadronic;
    P.lab_frame = d->lab_frame;
    P.kappa = nd[0].kind == PS_NODE_TCHAIN ? nd[0].n_children - 1 : 0;
    P.S = d->s_beam;
    P.sqrt_s = d->sqrt_s;
    P.a = d->a_shift;
    P.shat_M = d->shat_mass;
    P.shat_G = d->shat_width;
    P.shat_nu = d->shat_nu;
    P.t_nu = d->t_nu;
    P.ts_nu = d->ts_nu;
    P.vdims = d->vegas_dims;
    P.vbins = d->vegas_bins;
    double mleaf = 0.0;
    for (int j = 0; j < d->n_nodes; ++j) {
        InvNode& q = P.node[j];
        q.kind = nd[j].kind;
        q.nch = nd[j].n_children;
        q.leaf = nd[j].leaf_index;
        for (int k = 0; k < nd[j].n_children; ++k) q.child[k] = nd[j].children[k];
        unsigned m = 0;
        leaves_of(d, j, &m);
        q.mask = m;
        q.mass = nd[j].mass;
        q.M = nd[j].prop_mass;
        q.G = nd[j].prop_width;
        q.nu = nd[j].nu;
        if (nd[j].kind == PS_NODE_LEAF) mleaf += nd[j].mass;
    }
    P.mleaf = mleaf;
    std::vector<int> pre;
    preorder(d, 0, &pre);
    P.n_pre = static_cast<int>(pre.size());
    for (int i = 0; i < P.n_pre; ++i) P.pre[i] = pre[i];
    P.n_sorder = d->n_sorder;
    for (int i = 0; i < d->n_sorder; ++i) P.sorder[i] = d->sorder[i];
    // dimension layout (as the forward builder)
    for (int j = 0; j < kInvNodes; ++j) P.d_s[j] = P.d_dphi[j] = P.d_dth[j] = -1;
    int idx = 0;
    P.d_shat = P.d_x = -1;
    if (d->hadronic) P.d_shat = idx++;
    for (int i = 0; i < d->n_sorder; ++i) P.d_s[d->sorder[i]] = idx++;
    for (int i = 1; i < P.kappa; ++i) P.d_ts[i] = idx++;
    if (d->hadronic) P.d_x = idx++;
    for (int i = 1; i <= P.kappa; ++i) {
        P.d_tphi[i] = idx++;
        P.d_tt[i] = idx++;
    }
    for (int j : pre) {
        P.d_dphi[j] = idx++;
        P.d_dth[j] = idx++;
    }
    P.d = idx;
    // t-chain order (legs taken inwards from side A or B)
    if (P.kappa > 0) {
        int left = 0, right = P.kappa;
        for (int i = 1; i < P.kappa; ++i) {
            if (d->tside[i] == 0) {
                P.order[i] = left++;
                P.side[i] = 0;
            } else {
                P.order[i] = right--;
                P.side[i] = 1;
            }
        }
        P.order[P.kappa] = left;
        P.order[P.kappa + 1] = right;
    }
    // s-order bounds recipe
    std::vector<char> sampled(d->n_nodes, 0);
    sampled[0] = 1;
    int nid = 0;
    auto push = [&](int id) {
        if (nid >= kInvIds) throw PS_ERR_CAPACITY;
        P.ids[nid++] = id;
    };
    std::function<void(int, double*)> min_mass = [&](int j, double* c) {
        if (nd[j].kind == PS_NODE_LEAF) { *c += nd[j].mass; return; }
        if (sampled[j]) {
            if (j == 0 && !d->hadronic) *c += d->sqrt_s;
            else push(j);
            return;
        }
        for (int k = 0; k < nd[j].n_children; ++k) min_mass(nd[j].children[k], c);
    };
    try {
        for (int i = 0; i < d->n_sorder; ++i) {
            int j = d->sorder[i];
            P.lo_beg[i] = nid;
            P.lo_c[i] = 0.0;
            min_mass(j, &P.lo_c[i]);
            P.off_beg[i] = nid;
            P.off_c[i] = 0.0;
            int cur = j;
            for (;;) {
                int p = parent[cur];
                for (int k = 0; k < nd[p].n_children; ++k)
                    if (nd[p].children[k] != cur) min_mass(nd[p].children[k], &P.off_c[i]);
                if (sampled[p]) {
                    P.top[i] = p;
                    break;
                }
                cur = p;
            }
            P.lo_beg[i + 1] = nid;  // the end of this step's off list
            sampled[j] = 1;
        }
    } catch (int code) {
        *err = "inverse plan: too many bound terms";
        return code;
    }
    // SDE propagators
    std::vector<Prop> props = sde_props(d);
    if (static_cast<int>(props.size()) > kInvProps) {
        *err = "inverse plan: too many propagators";
        return PS_ERR_CAPACITY;
    }
    P.n_prop = static_cast<int>(props.size());
    for (int k = 0; k < P.n_prop; ++k) {
        P.pkind[k] = props[k].kind;
        P.pmask[k] = props[k].mask;
        P.pM[k] = props[k].M;
        P.pG[k] = props[k].G;
    }
    *plan = P;
    return PS_OK;
}
}  // namespace ps

extern "C" int ps_channel_dims(const ps_channel_desc* ch, int* n_random) {
    if (!ch || !n_random) return fail(PS_ERR_INVALID_ARGUMENT, "ps_channel_dims: null argument");
    std::string why;
    if (!validate_desc(ch, &why)) return fail(PS_ERR_GRAPH, "channel description: " + why);
    *n_random = random_dims(ch);
    return PS_OK;
}

extern "C" int ps_graph_build_channel(const ps_channel_desc* ch, int n_ch, int which, ps_graph* out) {
    if (!ch || !out || n_ch < 1 || n_ch > ps::kMaxChannels || which < 0 || which >= n_ch)
        return fail(PS_ERR_INVALID_ARGUMENT, "ps_graph_build_channel: bad arguments");
    std::string why;
    for (int c = 0; c < n_ch; ++c)
        if (!validate_desc(&ch[c], &why)) return fail(PS_ERR_GRAPH, "channel " + std::to_string(c) + ": " + why);
    int d = random_dims(&ch[which]);
    if (ch[which].vegas_dims > d) return fail(PS_ERR_GRAPH, "more VEGAS dimensions than random dimensions");
    ps_graph g;
    int st = ps_graph_create(d, &g);
    if (st != PS_OK) return st;
    try {
        build(ch, n_ch, which, g);
    } catch (int code) {
        ps_graph_free(g);
        return code;
    }
    *out = g;
    return PS_OK;
}

// ===================================================================== programs
struct ps_program_s {
    int device = 0;
    int n_ch = 0;
    int block = 128;
    int sm_count = 0;
    int grid_ctas = 0;
    size_t smem = 0;
    ps_options opt{};
    std::vector<Compiled> ch;
    std::vector<int> code_off, imm_off, grid_off, hist_off;
    int max_code = 0, max_imm = 0, max_grid = 0, max_slots = 0;
    std::vector<double> h_grid;
    int32_t* d_code = nullptr;
    double* d_imm = nullptr;
    double* d_grid = nullptr;
    double* d_stats = nullptr;
    double* d_hist = nullptr;
    double* d_hist_part = nullptr;    // training: per-(channel, chunk) partial histograms
    int hist_stride = 0;              // doubles per partial histogram (largest dims x bins)
    unsigned long long* d_status = nullptr;
    int32_t* d_stats_mode = nullptr;  // nonzero: reductions add into d_stats (ps_stats_accumulate)
    double* h_stats = nullptr;        // host-mapped pinned copy of d_stats (read-back of ps_stats)
    double* h_stats_dev = nullptr;    // its device address
    size_t hist_total = 0;
    bool training = false;
    void* jit_fn = nullptr;  // the compiled kernel (PS_PROGRAM_JIT), else the interpreter runs
    size_t jit_smem = 0;
    int jit_grid = 0;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return PS_OK;
    return fail(PS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void free_device(ps_program p) {
    cudaFree(p->d_code);
    cudaFree(p->d_imm);
    cudaFree(p->d_grid);
    cudaFree(p->d_stats);
    cudaFree(p->d_hist);
    cudaFree(p->d_hist_part);
    cudaFree(p->d_status);
    cudaFree(p->d_stats_mode);
    if (p->h_stats) cudaFreeHost(p->h_stats);
}

int64_t tiles_of(int64_t n, int block) { return (n + block - 1) / block; }

// The map launch of a program: its compiled kernel, else the interpreter.
int launch_program_map(ps_program p, const ps::LaunchParams& lp, void* stream, std::string* err) {
    if (p->jit_fn) {
        const int grid = static_cast<int>(std::min<int64_t>(std::max<int64_t>(lp.n_tiles, 1), p->jit_grid));
        return ps::jit_launch(p->jit_fn, lp, grid, p->jit_smem, stream, err);
    }
    const int grid = static_cast<int>(std::min<int64_t>(std::max<int64_t>(lp.n_tiles, 1), p->grid_ctas));
    return ps::launch_map(lp, grid, p->smem, stream, err);
}

// Fills the launch description shared by ps_generate and ps_map.
int fill_launch(ps_program p, const int* chans, const int64_t* counts, int n, const ps_out_buffers* out,
                void* workspace, size_t ws_bytes, ps::LaunchParams* lp) {
    std::memset(lp, 0, sizeof *lp);
    lp->n_ch = n;
    lp->block = p->block;
    lp->smem_code_ints = p->max_code;
    lp->smem_imm = p->max_imm;
    lp->smem_grid = p->max_grid;
    lp->smem_slots = p->max_slots;
    lp->code = p->d_code;
    lp->imm = p->d_imm;
    lp->grid = p->d_grid;
    int64_t tiles = 0, cols = 0;
    for (int k = 0; k < n; ++k) {
        int c = chans[k];
        if (counts[k] < 0) return fail(PS_ERR_INVALID_ARGUMENT, "negative event count");
        ps::ChannelLaunch& L = lp->ch[k];
        const Compiled& C = p->ch[c];
        L.code_off = p->code_off[c];
        L.code_len = static_cast<int32_t>(C.code.size());
        L.imm_off = p->imm_off[c];
        L.imm_len = static_cast<int32_t>(C.imm.size());
        L.grid_off = p->grid_off[c];
        L.vdims = C.vegas_dims;
        L.vbins = C.vegas_dims > 0 ? (p->grid_off[c + 1] - p->grid_off[c]) / C.vegas_dims - 1 : 1;
        L.n_slots = C.n_slots;
        L.n_random = C.n_random;
        L.hist_off = p->hist_off[c];
        L.channel = c;
        L.n_events = counts[k];
        L.col_off = cols;
        L.tile_begin = tiles;
        L.ev_offset = 0;
        cols += counts[k];
        tiles += tiles_of(counts[k], p->block);
    }
    lp->n_tiles = tiles;
    size_t need = static_cast<size_t>(tiles) * 4 * sizeof(double);
    if (tiles > 0 && (!workspace || ws_bytes < need))
        return fail(PS_ERR_INVALID_ARGUMENT, "workspace too small: need " + std::to_string(need) + " bytes");
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
        return fail(PS_ERR_INVALID_ARGUMENT, "workspace must be 256-byte aligned");
    lp->tile_partials = static_cast<double*>(workspace);
    lp->status = p->d_status;
    lp->stats_mode = p->d_stats_mode;
    lp->mixed = p->opt.precision == PS_PRECISION_MIXED ? 1 : 0;
    lp->hist = (p->training && p->hist_total > 0) ? p->d_hist : nullptr;
    if (lp->hist && tiles > 0 && (!out || !out->weight))
        return fail(PS_ERR_INVALID_ARGUMENT, "VEGAS training reads the weights: the weight output is required");
    if (out) {
        const Compiled& C0 = p->ch[chans[0]];
        if (C0.n_momenta_out > 0 && out->momenta && out->ld < cols)
            return fail(PS_ERR_INVALID_ARGUMENT, "ld smaller than the number of events");
        lp->mom = out->momenta;
        lp->x1 = out->x1;
        lp->x2 = out->x2;
        lp->w = out->weight;
        lp->alpha = out->alpha;
        lp->ld = out->ld;
        uintptr_t bad = 0;
        for (const void* q : {static_cast<const void*>(out->momenta), static_cast<const void*>(out->x1),
                              static_cast<const void*>(out->x2), static_cast<const void*>(out->weight),
                              static_cast<const void*>(out->alpha)})
            bad |= reinterpret_cast<uintptr_t>(q) % 16;
        if (bad) return fail(PS_ERR_INVALID_ARGUMENT, "output buffers must be 16-byte aligned");
    }
    return PS_OK;
}

}  // namespace

extern "C" {

int ps_program_create(const ps_graph* graphs, int n_ch, const ps_options* opt, int device, ps_program* out) {
    if (!graphs || !out || n_ch < 1 || n_ch > ps::kMaxChannels)
        return fail(PS_ERR_INVALID_ARGUMENT, "ps_program_create: bad arguments");
    for (int c = 0; c < n_ch; ++c)
        if (!graphs[c]) return fail(PS_ERR_INVALID_ARGUMENT, "ps_program_create: null graph");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(PS_ERR_NO_DEVICE, "no CUDA device available");
    }
    if (device < 0 || device >= ndev) return fail(PS_ERR_INVALID_ARGUMENT, "device index out of range");
    ps_program p = new (std::nothrow) ps_program_s;
    if (!p) return fail(PS_ERR_CAPACITY, "out of host memory");
    p->device = device;
    p->n_ch = n_ch;
    if (opt) p->opt = *opt;
    p->block = p->opt.block_threads > 0 ? p->opt.block_threads : 128;
    // the interpreter keeps a CTA's slot files in shared memory (at most 256 threads); a compiled
    // program keeps them in registers and may run 512-thread CTAs
    const bool jit = (p->opt.flags & PS_PROGRAM_JIT) != 0;
    if (p->block % 32 != 0 || p->block > (jit ? 512 : 256)) {
        delete p;
        return fail(PS_ERR_INVALID_ARGUMENT, jit ? "block_threads must be a multiple of 32 and at most 512"
                                                 : "block_threads must be a multiple of 32 and at most 256");
    }
    if (p->opt.precision != PS_PRECISION_F64 && p->opt.precision != PS_PRECISION_MIXED) {
        delete p;
        return fail(PS_ERR_INVALID_ARGUMENT, "unsupported precision mode");
    }
    p->ch.resize(n_ch);
    std::vector<int32_t> code;
    std::vector<double> imm;
    for (int c = 0; c < n_ch; ++c) {
        std::string err;
        int st = ps::compile_graph(graphs[c]->g, &p->ch[c], &err);
        if (st != PS_OK) {
            delete p;
            return fail(st, "channel " + std::to_string(c) + ": " + err);
        }
        const Compiled& C = p->ch[c];
        if (C.n_momenta_out != p->ch[0].n_momenta_out || C.has_x1 != p->ch[0].has_x1 || C.has_alpha != p->ch[0].has_alpha) {
            delete p;
            return fail(PS_ERR_GRAPH, "all channels of a program must declare the same outputs");
        }
        p->code_off.push_back(static_cast<int>(code.size()));
        code.insert(code.end(), C.code.begin(), C.code.end());
        p->imm_off.push_back(static_cast<int>(imm.size()));
        imm.insert(imm.end(), C.imm.begin(), C.imm.end());
        p->max_code = std::max(p->max_code, static_cast<int>(C.code.size()));
        p->max_imm = std::max(p->max_imm, static_cast<int>(C.imm.size()));
        p->max_slots = std::max(p->max_slots, C.n_slots);
    }
    // default VEGAS grids: identity with 64 bins.  A CTA's staged-grid region holds the azimuth
    // table, then the grid's edges and bin widths.
    int goff = 0, hoff = 0;
    p->max_grid = ps::kTrigDoubles;
    for (int c = 0; c < n_ch; ++c) {
        p->grid_off.push_back(goff);
        p->hist_off.push_back(hoff);
        int dv = p->ch[c].vegas_dims;
        if (dv > 0) {
            const int bins = 64;
            for (int j = 0; j < dv; ++j)
                for (int k = 0; k <= bins; ++k) p->h_grid.push_back(static_cast<double>(k) / bins);
            goff += dv * (bins + 1);
            hoff += dv * bins;
            p->max_grid = std::max(p->max_grid, ps::kTrigDoubles + dv * (2 * bins + 1));
        }
    }
    p->grid_off.push_back(goff);
    p->hist_off.push_back(hoff);
    p->hist_total = static_cast<size_t>(hoff);
    if (p->h_grid.empty()) p->h_grid.push_back(0.0);

    DeviceGuard dg(device);
    if (!dg.ok) { delete p; return fail(PS_ERR_CUDA, "cudaSetDevice failed"); }
    cudaDeviceProp prop;
    int st = cuda_check(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
    if (st != PS_OK) { delete p; return st; }
    p->sm_count = prop.multiProcessorCount;
    st = cuda_check(cudaMalloc(&p->d_code, code.size() * sizeof(int32_t)), "cudaMalloc code");
    if (st == PS_OK) st = cuda_check(cudaMalloc(&p->d_imm, imm.size() * sizeof(double)), "cudaMalloc imm");
    if (st == PS_OK) st = cuda_check(cudaMalloc(&p->d_grid, 2 * p->h_grid.size() * sizeof(double)), "cudaMalloc grid");
    if (st == PS_OK) st = cuda_check(cudaMalloc(&p->d_stats, 5 * n_ch * sizeof(double)), "cudaMalloc stats");
    if (st == PS_OK) st = cuda_check(cudaMalloc(&p->d_hist, std::max<size_t>(p->hist_total, 1) * sizeof(double)), "cudaMalloc hist");
    if (st == PS_OK) st = cuda_check(cudaMalloc(&p->d_status, 4 * sizeof(unsigned long long)), "cudaMalloc status");
    if (st == PS_OK) st = cuda_check(cudaMalloc(&p->d_stats_mode, sizeof(int32_t)), "cudaMalloc stats mode");
    if (st == PS_OK)
        st = cuda_check(cudaHostAlloc(&p->h_stats, 5 * n_ch * sizeof(double), cudaHostAllocMapped), "cudaHostAlloc stats");
    if (st == PS_OK) st = cuda_check(cudaHostGetDevicePointer(&p->h_stats_dev, p->h_stats, 0), "mapped stats");
    if (st == PS_OK) st = cuda_check(cudaMemcpy(p->d_code, code.data(), code.size() * sizeof(int32_t), cudaMemcpyHostToDevice), "upload code");
    if (st == PS_OK) st = cuda_check(cudaMemcpy(p->d_imm, imm.data(), imm.size() * sizeof(double), cudaMemcpyHostToDevice), "upload imm");
    if (st == PS_OK) st = cuda_check(cudaMemcpy(p->d_grid, p->h_grid.data(), p->h_grid.size() * sizeof(double), cudaMemcpyHostToDevice), "upload grid");
    if (st == PS_OK) st = cuda_check(cudaMemset(p->d_stats, 0, 5 * n_ch * sizeof(double)), "memset stats");
    if (st == PS_OK) st = cuda_check(cudaMemset(p->d_hist, 0, std::max<size_t>(p->hist_total, 1) * sizeof(double)), "memset hist");
    if (st == PS_OK) st = cuda_check(cudaMemset(p->d_status, 0, 4 * sizeof(unsigned long long)), "memset status");
    if (st == PS_OK) st = cuda_check(cudaMemset(p->d_stats_mode, 0, sizeof(int32_t)), "memset stats mode");
    if (st != PS_OK) { free_device(p); delete p; return st; }

    ps::LaunchParams lp;
    std::memset(&lp, 0, sizeof lp);
    lp.block = p->block;
    lp.smem_code_ints = p->max_code;
    lp.smem_imm = p->max_imm;
    lp.smem_grid = p->max_grid;
    lp.smem_slots = p->max_slots;
    lp.mixed = p->opt.precision == PS_PRECISION_MIXED ? 1 : 0;  // the mixed kernel also stages float immediates
    p->smem = ps::smem_bytes_for(lp);
    std::string err;
    if (p->block <= 256) {  // the interpreter's launch shape (a compiled program never launches it)
        if (p->smem > static_cast<size_t>(prop.sharedMemPerBlockOptin)) {
            free_device(p);
            delete p;
            return fail(PS_ERR_CAPACITY, "channel needs " + std::to_string(p->smem) + " bytes of shared memory per CTA");
        }
        int per_sm = 0;
        st = ps::max_ctas_per_sm(p->block, p->smem, p->opt.precision == PS_PRECISION_MIXED, &per_sm, &err);
        if (st != PS_OK || per_sm < 1) {
            free_device(p);
            delete p;
            return fail(st != PS_OK ? st : PS_ERR_CAPACITY, st != PS_OK ? err : "kernel does not fit on an SM");
        }
        int want = p->opt.ctas_per_sm > 0 ? p->opt.ctas_per_sm : 4;
        p->grid_ctas = p->sm_count * std::min(per_sm, want);
    }
    if (p->opt.flags & PS_PROGRAM_JIT) {  // the compiled kernel: VEGAS grid and reduction scratch in shared memory
        // a requested CTA count also caps the compiled kernel's registers so that many CTAs fit
        const int min_blocks = std::min(p->opt.ctas_per_sm, 2048 / p->block);
        st = ps::jit_prepare(p->ch, p->block, min_blocks, p->opt.precision == PS_PRECISION_MIXED, device, &p->jit_fn,
                             &err);
        int jit_per_sm = 0;
        p->jit_smem = (static_cast<size_t>(p->max_grid) + 4 * (p->block / 32)) * sizeof(double);
        if (st == PS_OK) st = ps::jit_occupancy(p->jit_fn, p->block, p->jit_smem, &jit_per_sm);
        if (st != PS_OK || jit_per_sm < 1) {
            free_device(p);
            delete p;
            return fail(st != PS_OK ? st : PS_ERR_CAPACITY, st != PS_OK ? err : "compiled kernel does not fit on an SM");
        }
        const int jit_want = p->opt.ctas_per_sm > 0 ? p->opt.ctas_per_sm : 16;
        p->jit_grid = p->sm_count * std::min(jit_per_sm, jit_want);
    }
    *out = p;
    return PS_OK;
}

int ps_program_set_vegas(ps_program p, int ch, int dims, int bins, const double* edges) {
    if (!p || !edges || ch < 0 || ch >= p->n_ch) return fail(PS_ERR_INVALID_ARGUMENT, "ps_program_set_vegas: bad arguments");
    const Compiled& C = p->ch[ch];
    if (dims != C.vegas_dims || bins < 1) return fail(PS_ERR_INVALID_ARGUMENT, "grid dimensions differ from the channel's VEGAS op");
    int cur_bins = (p->grid_off[ch + 1] - p->grid_off[ch]) / dims - 1;
    if (bins != cur_bins) return fail(PS_ERR_INVALID_ARGUMENT, "the number of bins is fixed at 64");
    for (int j = 0; j < dims; ++j) {
        const double* e = edges + j * (bins + 1);
        if (e[0] != 0.0 || e[bins] != 1.0) return fail(PS_ERR_INVALID_ARGUMENT, "grid rows must run from 0 to 1");
        for (int k = 0; k < bins; ++k)
            if (!(e[k + 1] >= e[k])) return fail(PS_ERR_INVALID_ARGUMENT, "grid edges must be non-decreasing");
    }
    std::memcpy(p->h_grid.data() + p->grid_off[ch], edges, sizeof(double) * dims * (bins + 1));
    DeviceGuard dg(p->device);
    return cuda_check(cudaMemcpy(p->d_grid + p->grid_off[ch], edges, sizeof(double) * dims * (bins + 1),
                                 cudaMemcpyHostToDevice), "upload grid");
}

int ps_program_get_vegas(ps_program p, int ch, int dims, int bins, double* edges) {
    if (!p || !edges || ch < 0 || ch >= p->n_ch || dims != p->ch[ch].vegas_dims)
        return fail(PS_ERR_INVALID_ARGUMENT, "ps_program_get_vegas: bad arguments");
    int cur_bins = dims > 0 ? (p->grid_off[ch + 1] - p->grid_off[ch]) / dims - 1 : 0;
    if (bins != cur_bins) return fail(PS_ERR_INVALID_ARGUMENT, "bins differ");
    std::memcpy(edges, p->h_grid.data() + p->grid_off[ch], sizeof(double) * dims * (bins + 1));
    return PS_OK;
}

int ps_workspace_size(ps_program p, const int64_t* events, size_t* bytes) {
    if (!p || !events || !bytes) return fail(PS_ERR_INVALID_ARGUMENT, "ps_workspace_size: bad arguments");
    int64_t tiles = 0;
    for (int c = 0; c < p->n_ch; ++c) {
        if (events[c] < 0) return fail(PS_ERR_INVALID_ARGUMENT, "negative event count");
        tiles += tiles_of(events[c], p->block);
    }
    *bytes = std::max<size_t>(256, (static_cast<size_t>(tiles) * 4 * sizeof(double) + 255) / 256 * 256);
    return PS_OK;
}

int ps_generate(ps_program p, const int64_t* events, uint64_t seed, uint64_t event_offset, const ps_out_buffers* out,
                void* workspace, size_t ws_bytes, void* stream) {
    if (!p || !events || !out) return fail(PS_ERR_INVALID_ARGUMENT, "ps_generate: bad arguments");
    std::vector<int> chans(p->n_ch);
    for (int c = 0; c < p->n_ch; ++c) chans[c] = c;
    ps::LaunchParams lp;
    int st = fill_launch(p, chans.data(), events, p->n_ch, out, workspace, ws_bytes, &lp);
    if (st != PS_OK) return st;
    for (int c = 0; c < p->n_ch; ++c) lp.ch[c].ev_offset = static_cast<int64_t>(event_offset);
    lp.r = nullptr;
    lp.seed = seed;
    DeviceGuard dg(p->device);
    std::string err;
    if (lp.n_tiles > 0) {
        st = launch_program_map(p, lp, stream, &err);
        if (st != PS_OK) return fail(st, err);
    }
    st = ps::launch_reduce(lp, p->d_stats, stream, &err);
    if (st == PS_OK && lp.n_tiles > 0) st = ps::launch_hist(lp, p->d_hist_part, p->hist_stride, stream, &err);
    if (st != PS_OK) return fail(st, err);
    return PS_OK;
}

}  // extern "C"

struct ps_exec_s {
    ps_program p = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t map_node = nullptr, reduce_node = nullptr;
    std::vector<cudaGraphNode_t> hist_nodes;  // VEGAS training histogram kernels (training programs)
    ps::LaunchParams lp;
    double* stats = nullptr;
    int grid = 0;
};

extern "C" {

int ps_exec_create(ps_program p, const int64_t* events, const ps_out_buffers* out, void* workspace,
                   size_t ws_bytes, ps_exec* exec_out) {
    if (!p || !events || !out || !exec_out) return fail(PS_ERR_INVALID_ARGUMENT, "ps_exec_create: bad arguments");
    ps_exec e = new (std::nothrow) ps_exec_s;
    if (!e) return fail(PS_ERR_CAPACITY, "out of host memory");
    e->p = p;
    std::vector<int> chans(p->n_ch);
    for (int c = 0; c < p->n_ch; ++c) chans[c] = c;
    int st = fill_launch(p, chans.data(), events, p->n_ch, out, workspace, ws_bytes, &e->lp);
    if (st != PS_OK) { delete e; return st; }
    e->lp.r = nullptr;
    e->stats = p->d_stats;
    e->grid = static_cast<int>(
        std::min<int64_t>(std::max<int64_t>(e->lp.n_tiles, 1), p->jit_fn ? p->jit_grid : p->grid_ctas));
    DeviceGuard dg(p->device);
    cudaStream_t cs;
    st = cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
    if (st != PS_OK) { delete e; return st; }
    std::string err;
    st = cuda_check(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    if (st == PS_OK && e->lp.n_tiles > 0) st = launch_program_map(p, e->lp, cs, &err);
    if (st == PS_OK) st = ps::launch_reduce(e->lp, e->stats, cs, &err);
    if (st == PS_OK && e->lp.n_tiles > 0) st = ps::launch_hist(e->lp, p->d_hist_part, p->hist_stride, cs, &err);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st != PS_OK) { if (g) cudaGraphDestroy(g); delete e; return fail(st, err.empty() ? t_err : err); }
    st = cuda_check(ce, "cudaStreamEndCapture");
    if (st != PS_OK) { delete e; return st; }
    e->graph = g;
    size_t n = 0;
    cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(g, nodes.data(), &n);
    for (size_t k = 0; k < n; ++k) {
        cudaGraphNodeType t;
        cudaGraphNodeGetType(nodes[k], &t);
        if (t != cudaGraphNodeTypeKernel) continue;
        if (p->jit_fn && ps::jit_node_runs(nodes[k], p->jit_fn)) {
            e->map_node = nodes[k];  // a compiled program's kernel, launched through the driver
            continue;
        }
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(nodes[k], &kp) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (ps::is_reduce_kernel(kp.func)) e->reduce_node = nodes[k];
        else if (ps::is_hist_kernel(kp.func)) e->hist_nodes.push_back(nodes[k]);
        else if (!p->jit_fn) e->map_node = nodes[k];
    }
    if (e->lp.n_tiles > 0 && !e->map_node) {
        cudaGraphDestroy(g);
        delete e;
        return fail(PS_ERR_CUDA, "ps_exec_create: the captured graph has no map kernel node");
    }
    st = cuda_check(cudaGraphInstantiate(&e->exec, g, 0), "cudaGraphInstantiate");
    if (st != PS_OK) { cudaGraphDestroy(g); delete e; return st; }
    *exec_out = e;
    return PS_OK;
}

int ps_exec_launch(ps_exec e, uint64_t seed, uint64_t event_offset, void* stream) {
    if (!e) return fail(PS_ERR_INVALID_ARGUMENT, "ps_exec_launch: null executor");
    e->lp.seed = seed;
    for (int c = 0; c < e->lp.n_ch; ++c) e->lp.ch[c].ev_offset = static_cast<int64_t>(event_offset);
    DeviceGuard dg(e->p->device);
    if (e->map_node && e->p->jit_fn) {
        std::string err;
        int st = ps::jit_node_set(e->exec, e->map_node, e->p->jit_fn, e->lp, e->grid, e->p->jit_smem, &err);
        if (st != PS_OK) return fail(st, err);
    } else if (e->map_node) {
        cudaKernelNodeParams kp;
        int st = cuda_check(cudaGraphKernelNodeGetParams(e->map_node, &kp), "cudaGraphKernelNodeGetParams");
        if (st != PS_OK) return st;
        void* args[1] = {&e->lp};
        kp.kernelParams = args;
        kp.extra = nullptr;
        st = cuda_check(cudaGraphExecKernelNodeSetParams(e->exec, e->map_node, &kp), "cudaGraphExecKernelNodeSetParams");
        if (st != PS_OK) return st;
    }
    for (cudaGraphNode_t hn : e->hist_nodes) {  // the histogram kernels read the same seed and offsets
        cudaKernelNodeParams kp;
        int st = cuda_check(cudaGraphKernelNodeGetParams(hn, &kp), "cudaGraphKernelNodeGetParams");
        if (st != PS_OK) return st;
        double* part = e->p->d_hist_part;
        int stride = e->p->hist_stride;
        void* args[3] = {&e->lp, &part, &stride};
        kp.kernelParams = args;
        kp.extra = nullptr;
        st = cuda_check(cudaGraphExecKernelNodeSetParams(e->exec, hn, &kp), "cudaGraphExecKernelNodeSetParams");
        if (st != PS_OK) return st;
    }
    int st = cuda_check(cudaGraphLaunch(e->exec, static_cast<cudaStream_t>(stream)), "cudaGraphLaunch");
    if (st == PS_OK) ps::count_launches((e->map_node ? 2 : 1) + static_cast<int>(e->hist_nodes.size()));
    return st;
}

int ps_exec_free(ps_exec e) {
    if (!e) return PS_OK;
    {
        DeviceGuard dg(e->p->device);
        if (e->exec) cudaGraphExecDestroy(e->exec);
        if (e->graph) cudaGraphDestroy(e->graph);
    }
    delete e;
    return PS_OK;
}

int ps_generate_noalloc(ps_program p, const int64_t* events, uint64_t seed, uint64_t event_offset,
                        const ps_out_buffers* out, void* stream) {
    if (!p || !events || !out) return fail(PS_ERR_INVALID_ARGUMENT, "ps_generate_noalloc: bad arguments");
    int64_t tiles = 0;
    for (int c = 0; c < p->n_ch; ++c) {
        if (events[c] < 0) return fail(PS_ERR_INVALID_ARGUMENT, "ps_generate_noalloc: negative event count");
        tiles += tiles_of(events[c], p->block);
    }
    if (tiles > ps::kNoallocTiles)
        return fail(PS_ERR_CAPACITY, "ps_generate_noalloc: " + std::to_string(tiles) + " tiles of " +
                                         std::to_string(p->block) + " events exceed the fixed scratch of " +
                                         std::to_string(ps::kNoallocTiles) + " tiles; use ps_generate with a workspace");
    DeviceGuard dg(p->device);
    if (!dg.ok) return fail(PS_ERR_CUDA, "cudaSetDevice failed");
    void* scratch = nullptr;
    size_t bytes = 0;
    std::string err;
    int st = ps::noalloc_scratch(p->device, &scratch, &bytes, &err);
    if (st != PS_OK) return fail(st, err);
    return ps_generate(p, events, seed, event_offset, out, scratch, bytes, stream);
}

int ps_map(ps_program p, int ch, int64_t batch, const double* r, int64_t ld_r, const ps_out_buffers* out,
           void* workspace, size_t ws_bytes, void* stream) {
    if (!p || !out || ch < 0 || ch >= p->n_ch || batch < 0 || (batch > 0 && !r) || ld_r < batch)
        return fail(PS_ERR_INVALID_ARGUMENT, "ps_map: bad arguments");
    ps::LaunchParams lp;
    int st = fill_launch(p, &ch, &batch, 1, out, workspace, ws_bytes, &lp);
    if (st != PS_OK) return st;
    lp.r = r;
    lp.ld_r = ld_r;
    DeviceGuard dg(p->device);
    std::string err;
    if (lp.n_tiles > 0) {
        st = launch_program_map(p, lp, stream, &err);
        if (st != PS_OK) return fail(st, err);
    }
    st = ps::launch_reduce(lp, p->d_stats + 5 * ch, stream, &err);
    if (st == PS_OK && lp.n_tiles > 0) st = ps::launch_hist(lp, p->d_hist_part, p->hist_stride, stream, &err);
    if (st != PS_OK) return fail(st, err);
    return PS_OK;
}

int ps_inverse_map(ps_program p, int ch, const ps_channel_desc* desc, int64_t batch, const double* momenta,
                   int64_t ld_m, const double* x1, const double* x2, double* r, int64_t ld_r, double* P,
                   void* stream) {
    if (!p || !desc || ch < 0 || ch >= p->n_ch || batch < 0 || ld_m < batch || ld_r < batch ||
        (batch > 0 && (!momenta || !r)))
        return fail(PS_ERR_INVALID_ARGUMENT, "ps_inverse_map: bad arguments");
    ps::InvPlan plan;
    std::string err;
    int st = ps::build_inverse_plan(desc, &plan, &err);
    if (st != PS_OK) return fail(st, err);
    const ps::Compiled& C = p->ch[ch];
    if (plan.d != C.n_random || plan.vdims != C.vegas_dims)
        return fail(PS_ERR_INVALID_ARGUMENT, "ps_inverse_map: the description does not match the program's channel");
    if (plan.hadronic && batch > 0 && (!x1 || !x2))
        return fail(PS_ERR_INVALID_ARGUMENT, "ps_inverse_map: a hadronic channel needs x1 and x2");
    if (plan.n + 2 > ps::kMaxOutMomenta + 2 || plan.n_nodes > ps::kInvNodes)
        return fail(PS_ERR_CAPACITY, "ps_inverse_map: channel too large");
    plan.vbins = C.vegas_dims > 0 ? (p->grid_off[ch + 1] - p->grid_off[ch]) / C.vegas_dims - 1 : 1;
    DeviceGuard dg(p->device);
    st = ps::launch_inverse(plan, batch, momenta, ld_m, x1, x2, p->d_grid + p->grid_off[ch], r, ld_r, P, stream,
                            &err);
    return st == PS_OK ? PS_OK : fail(st, err);
}

int ps_global_weights(int n_ch, int64_t batch, const double* J, int64_t ld_j, const double* P, int64_t ld_p,
                      const double* alpha, const double* x1, const double* x2, double pdf_alpha, double pdf_beta,
                      const double* f, double* w, void* stream) {
    if (n_ch < 1 || n_ch > ps::kMaxChannels || batch < 0 || !alpha || ld_j < batch ||
        (batch > 0 && (!J || !w || (!f && (!P || ld_p < batch)))) || ((x1 == nullptr) != (x2 == nullptr)))
        return fail(PS_ERR_INVALID_ARGUMENT, "ps_global_weights: bad arguments");
    for (int j = 0; j < n_ch; ++j)
        if (!(alpha[j] >= 0.0)) return fail(PS_ERR_INVALID_ARGUMENT, "ps_global_weights: negative channel weight");
    std::string err;
    int st = ps::launch_global_weights(n_ch, batch, J, ld_j, P, ld_p, alpha, x1, x2, pdf_alpha, pdf_beta, f, w,
                                       stream, &err);
    return st == PS_OK ? PS_OK : fail(st, err);
}

int ps_stats(ps_program p, ps_channel_stats* host, int n_ch, void* stream) {
    if (!p || !host || n_ch < 1 || n_ch > p->n_ch) return fail(PS_ERR_INVALID_ARGUMENT, "ps_stats: bad arguments");
    DeviceGuard dg(p->device);
    std::string err;
    int st = ps::launch_copy(p->h_stats_dev, p->d_stats, 5 * n_ch, stream, &err);
    if (st != PS_OK) return fail(st, err);
    st = cuda_check(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "stream sync");
    if (st != PS_OK) return st;
    const double* h = p->h_stats;
    for (int c = 0; c < n_ch; ++c) {
        host[c].n = h[5 * c];
        host[c].n_nonzero = h[5 * c + 1];
        host[c].sum_w = h[5 * c + 2];
        host[c].sum_w2 = h[5 * c + 3];
        host[c].max_w = h[5 * c + 4];
    }
    return PS_OK;
}

int ps_jit_check(const ps_graph* graphs, int n_ch, const ps_options* opt, char* log, size_t log_bytes) {
    if (!graphs || n_ch < 1 || n_ch > ps::kMaxChannels || (log_bytes > 0 && !log))
        return fail(PS_ERR_INVALID_ARGUMENT, "ps_jit_check: bad arguments");
    const bool mixed = opt && opt->precision == PS_PRECISION_MIXED;
    const int block = (opt && opt->block_threads > 0) ? opt->block_threads : 128;
    std::vector<Compiled> ch(n_ch);
    std::string err;
    for (int c = 0; c < n_ch; ++c) {
        if (!graphs[c]) return fail(PS_ERR_INVALID_ARGUMENT, "ps_jit_check: null graph");
        int st = ps::compile_graph(graphs[c]->g, &ch[c], &err);
        if (st != PS_OK) return fail(st, "channel " + std::to_string(c) + ": " + err);
    }
    std::vector<char> cubin;
    std::string lg;
    const int min_blocks = opt ? std::min(opt->ctas_per_sm, 2048 / block) : 0;
    int st = ps::jit_build(ch, block, min_blocks, mixed, &cubin, &lg);
    if (log_bytes > 0) {
        std::snprintf(log, log_bytes, "%s", lg.c_str());
    }
    if (st != PS_OK) return fail(st, "NVRTC: " + lg);
    return PS_OK;
}

int ps_stats_accumulate(ps_program p, int enable, void* stream) {
    if (!p) return fail(PS_ERR_INVALID_ARGUMENT, "ps_stats_accumulate: null program");
    DeviceGuard dg(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st = PS_OK;
    if (enable) st = cuda_check(cudaMemsetAsync(p->d_stats, 0, 5 * p->n_ch * sizeof(double), s), "zero stats");
    if (st == PS_OK) st = cuda_check(cudaMemsetAsync(p->d_stats_mode, enable ? 1 : 0, sizeof(int32_t), s), "stats mode");
    return st;
}

int ps_vegas_training(ps_program p, int enable) {
    if (!p) return fail(PS_ERR_INVALID_ARGUMENT, "ps_vegas_training: null program");
    if (enable && p->hist_total > 0 && !p->d_hist_part) {
        int stride = 0;
        for (int c = 0; c < p->n_ch; ++c) {
            const int dv = p->ch[c].vegas_dims;
            if (dv == 0) continue;
            const int bins = (p->grid_off[c + 1] - p->grid_off[c]) / dv - 1;
            if (dv > ps::kHistMaxDims || bins > 256 || dv * bins > ps::kHistThreads * ps::kHistEntries)
                return fail(PS_ERR_CAPACITY, "ps_vegas_training: VEGAS grid too large for the training histogram");
            stride = std::max(stride, dv * bins);
        }
        DeviceGuard dg(p->device);
        const size_t bytes = static_cast<size_t>(p->n_ch) * ps::kHistChunks * stride * sizeof(double);
        int st = cuda_check(cudaMalloc(&p->d_hist_part, bytes), "cudaMalloc training histogram");
        if (st != PS_OK) return st;
        p->hist_stride = stride;
    }
    p->training = enable != 0;
    return PS_OK;
}

int ps_vegas_histogram(ps_program p, int ch, double* hist, void* stream) {
    if (!p || !hist || ch < 0 || ch >= p->n_ch) return fail(PS_ERR_INVALID_ARGUMENT, "ps_vegas_histogram: bad arguments");
    int n = p->hist_off[ch + 1] - p->hist_off[ch];
    if (n == 0) return PS_OK;
    DeviceGuard dg(p->device);
    int st = cuda_check(cudaMemcpyAsync(hist, p->d_hist + p->hist_off[ch], n * sizeof(double), cudaMemcpyDeviceToHost,
                                        static_cast<cudaStream_t>(stream)), "copy histogram");
    if (st == PS_OK) st = cuda_check(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "stream sync");
    return st;
}

// VEGAS grid refinement of one dimension (Lepage 1978; the adaptive VEGAS sampling of
// Sec. 3.2.2).  The importance of a bin is the mean of its histogram entry and those of its
// neighbours inside the grid; the shares d_k of these means are damped to
// m_k = ((1 - d_k) / ln(1/d_k))^alpha.  Spread evenly across each old bin, m has a piecewise-linear
// cumulative M(x); the new edge j is the point where M reaches j/N of its total, found by a
// binary search over the old bins' cumulative ends.
static void rebin_row(const double* h, const double* e, double* out, int N, double alpha) {
    std::vector<double> imp(N), cum(N + 1, 0.0);
    double total = 0.0;
    for (int k = 0; k < N; ++k) {
        const int first = std::max(k - 1, 0), last = std::min(k + 1, N - 1);
        double s = 0.0;
        for (int i = first; i <= last; ++i) s += h[i];
        imp[k] = s / static_cast<double>(last - first + 1);
        total += imp[k];
    }
    if (!(total > 0.0)) {  // nothing was sampled (or the sums overflowed): keep the grid
        std::copy(e, e + N + 1, out);
        return;
    }
    for (int k = 0; k < N; ++k) {
        const double d = imp[k] / total;
        imp[k] = d <= 0.0 ? 0.0 : d >= 1.0 ? 1.0 : std::pow((1.0 - d) / -std::log(d), alpha);
        cum[k + 1] = cum[k] + imp[k];
    }
    out[0] = e[0];
    out[N] = e[N];
    for (int j = 1; j < N; ++j) {
        const double target = cum[N] * static_cast<double>(j) / static_cast<double>(N);
        // the first old bin whose cumulative end reaches the target holds the new edge
        const int k = std::min(static_cast<int>(std::lower_bound(cum.begin() + 1, cum.end(), target) - cum.begin()) - 1,
                               N - 1);
        const double u = imp[k] > 0.0 ? std::clamp((target - cum[k]) / imp[k], 0.0, 1.0) : 0.0;
        out[j] = e[k] + u * (e[k + 1] - e[k]);
    }
}

int ps_vegas_adapt(ps_program p, int ch, double alpha, void* stream) {
    if (!p || ch < 0 || ch >= p->n_ch) return fail(PS_ERR_INVALID_ARGUMENT, "ps_vegas_adapt: bad arguments");
    const int dv = p->ch[ch].vegas_dims;
    if (dv == 0) return PS_OK;
    const int N = (p->grid_off[ch + 1] - p->grid_off[ch]) / dv - 1;
    std::vector<double> h(static_cast<size_t>(dv) * N), ne(static_cast<size_t>(dv) * (N + 1));
    int st = ps_vegas_histogram(p, ch, h.data(), stream);
    if (st != PS_OK) return st;
    for (int j = 0; j < dv; ++j)
        rebin_row(h.data() + j * N, p->h_grid.data() + p->grid_off[ch] + j * (N + 1), ne.data() + j * (N + 1), N, alpha);
    st = ps_program_set_vegas(p, ch, dv, N, ne.data());
    if (st != PS_OK) return st;
    DeviceGuard dg(p->device);
    return cuda_check(cudaMemset(p->d_hist + p->hist_off[ch], 0, h.size() * sizeof(double)), "clear histogram");
}

int ps_status(ps_program p, int64_t* counters, int n, void* stream) {
    if (!p || !counters || n < 1 || n > 4) return fail(PS_ERR_INVALID_ARGUMENT, "ps_status: bad arguments");
    DeviceGuard dg(p->device);
    unsigned long long h[4];
    int st = cuda_check(cudaMemcpyAsync(h, p->d_status, sizeof h, cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)),
                        "copy status");
    if (st == PS_OK) st = cuda_check(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "stream sync");
    if (st != PS_OK) return st;
    for (int k = 0; k < n; ++k) counters[k] = static_cast<int64_t>(h[k]);
    return PS_OK;
}

int ps_status_reset(ps_program p, void* stream) {
    if (!p) return fail(PS_ERR_INVALID_ARGUMENT, "ps_status_reset: null program");
    DeviceGuard dg(p->device);
    return cuda_check(cudaMemsetAsync(p->d_status, 0, 4 * sizeof(unsigned long long), static_cast<cudaStream_t>(stream)),
                      "reset status");
}

int ps_program_free(ps_program p) {
    if (!p) return PS_OK;
    {
        DeviceGuard dg(p->device);
        free_device(p);
    }
    delete p;
    return PS_OK;
}

int64_t ps_launch_count(void) { return static_cast<int64_t>(ps::launch_count()); }

}  // extern "C"
