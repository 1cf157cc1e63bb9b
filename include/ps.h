/*
 * ps.h -- C ABI of the GB300 phase-space library.
 *
 * The library maps uniform random numbers to weighted collider events on an
 * sm_103a GPU: the data-parallel hot path of "MadSpace -- Event Generation for
 * the Era of GPUs and ML" (arXiv 2602.06895).  Its calls follow the paper's
 * compute-graph formulation (Sec. 3.1, Fig. compute_graph): a channel is an
 * ordered list of inputs (random numbers), instructions in static single
 * assignment form with inline immediate constants, and outputs.  A *program*
 * compiles the graphs of one or more channels for one device; a single fused
 * kernel then evaluates every instruction of an event in that event's own thread,
 * with intermediate values in shared memory and registers, and writes only the
 * outputs (SoA) and per-tile partial sums.
 *
 * Conventions (after the UMAMI interface of Sec. 3.3):
 *   - every function returns an int status: PS_OK (0) or a negative PS_ERR_*;
 *     nothing throws or aborts; ps_last_error() returns a thread-local message;
 *   - pointers named *_dev are device pointers owned by the caller; *_host are
 *     host pointers owned by the caller; the library owns graphs and programs
 *     (and their device constants) until the matching *_free call;
 *   - streams are passed as void* (a cudaStream_t; NULL = legacy default stream);
 *   - inputs are never modified (Sec. 3.1: operations consume immutable inputs).
 *
 * All floating point is IEEE binary64 unless a function says otherwise.
 */
#ifndef PS_H
#define PS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define PS_OK 0
#define PS_ERR_INVALID_ARGUMENT (-1) /* null handle/pointer, bad size, bad id      */
#define PS_ERR_GRAPH (-2)            /* malformed graph: arity, type, undefined id */
#define PS_ERR_CUDA (-3)             /* a CUDA runtime call failed                  */
#define PS_ERR_DEVICE_STATUS (-4)    /* the device status word reports a fault      */
#define PS_ERR_CAPACITY (-5)         /* a fixed limit of the library was exceeded   */
#define PS_ERR_NO_DEVICE (-6)        /* no usable CUDA device                       */

/* Message of the last error on the calling thread ("" if none). */
const char* ps_last_error(void);

/* Library version (major*10000 + minor*100 + patch). */
int ps_version(void);

/* ---------------------------------------------------------------- graphs */
typedef struct ps_graph_s* ps_graph;
typedef struct ps_program_s* ps_program;

/* Value types of graph values. */
#define PS_TYPE_SCALAR 0 /* one f64 per event          */
#define PS_TYPE_MOMENTUM 1 /* four f64 (E, px, py, pz) */

/* Argument of an instruction: a previously defined value, or an immediate f64. */
#define PS_ARG_VALUE 0
#define PS_ARG_IMM 1
typedef struct {
    int32_t kind; /* PS_ARG_VALUE or PS_ARG_IMM */
    int32_t id;   /* value id (PS_ARG_VALUE)    */
    double imm;   /* constant (PS_ARG_IMM)      */
} ps_arg;

/* Opcodes.  "(a, b) -> (c, d)" lists argument and result types: s = scalar,
 * p = momentum, i = must be immediate; "..." marks a variadic tail.  Paper
 * citations are sections / equations of arXiv 2602.06895. */
enum {
    /* VEGAS grid lookup (Sec. 3.2.2; Lepage 1978):
     * (s r_0, ..., s r_{k-1}) -> (s r'_0, ..., s r'_{k-1}, s J).  Uses the channel's grid
     * (ps_program_set_vegas); dimension j of the op uses grid row j. */
    PS_OP_VEGAS = 1,
    /* Power-law invariant map G_nu, Eqs. prop_stable_nu / prop_stable_nu1 (Sec. 2.2.1),
     * stable_invariant_nu of the example graph:
     * (s r, s|i m, i nu, s|i x_min, s|i x_max, i a) -> (s x, s J).  m <= 0 selects the
     * auxiliary mass m^2 = -a; nu = 1 is the logarithmic map.  J = dx/dr. */
    PS_OP_INVARIANT_NU = 2,
    /* Breit-Wigner map G_BW, Eq. prop_massive (Sec. 2.2.1):
     * (s r, i M, i Gamma, s|i x_min, s|i x_max [, i u1]) -> (s x, s J).  The optional u1 is
     * atan((x_min - M^2)/(M Gamma)), the lower angle, when x_min is a constant. */
    PS_OP_INVARIANT_BW = 3,
    /* r_to_x1x2, Eq. pdf_sampling (Sec. 2.2.2): (s r, s shat, i S) -> (s x1, s x2, s J),
     * J = -log(shat/S)/S.  With a fourth immediate argument (any value) it also returns
     * (s log x1, s log x2) = (r, 1 - r) log(shat/S). */
    PS_OP_R_TO_X1X2 = 4,
    /* com_p_in (Sec. 3.2): (s sqrt_shat) -> (p p_a, p p_b) along +-z. */
    PS_OP_COM_P_IN = 5,
    /* t_inv_min_max (Sec. 2.2.4, Eq. t_invariant_theta):
     * (s s, s|i mA^2, s|i mB^2, s|i m1, s|i m2) -> (s |t|_min, s |t|_max).
     * The block invariant s and the incoming invariant masses are passed as scalars
     * (the paper passes the momenta) so that they keep the precision they were sampled with. */
    PS_OP_T_INV_MIN_MAX = 6,
    /* two_to_two_particle_scattering_com (Sec. 2.2.4, Eqs. 2_to_2_mapping, ps2_phi_t):
     * (s r_phi, p pA, p pB, s |t|, s|i m1, s|i m2, s s, s|i mA^2, s|i mB^2) -> (p p1, p p2, s J),
     * J = 2 pi / (4 sqrt(lambda(s, mA^2, mB^2))). */
    PS_OP_TWO_TO_TWO_COM = 7,
    /* two_body_decay (Sec. 2.2.3, Eq. ps2_phi_theta), boosted to the frame of p0:
     * (s r_phi, s r_theta, s s0, s|i m1, s|i m2, p p0) -> (p p1, p p2, s J),
     * J = pi sqrt(lambda(s0, m1^2, m2^2)) / (2 s0). */
    PS_OP_TWO_BODY_DECAY = 8,
    /* the same decay with the parent at rest: (s r_phi, s r_theta, s s0, s|i m1, s|i m2)
     * -> (p p1, p p2, s J). */
    PS_OP_TWO_BODY_DECAY_COM = 9,
    /* boost_beam (Sec. 3.2): (p q_0, ..., p q_{k-1}, s x1, s x2) -> (p q'_0, ..., p q'_{k-1}):
     * the longitudinal boost with rapidity log(x1/x2)/2, E' +- p_z' = (E +- p_z) (x1/x2)^(+-1/2). */
    PS_OP_BOOST_BEAM = 10,
    /* reduce_product (Sec. 3.2): (s|i a_0, ...) -> (s a_0 a_1 ...), left to right. */
    PS_OP_REDUCE_PRODUCT = 11,
    /* cut_unphysical (Sec. 3.2): (s w, s x1, s x2, p q_0, ...) -> (s w').  w' = 0 if w or any
     * momentum component is not finite, or x1 or x2 is outside (0, 1]. */
    PS_OP_CUT_UNPHYSICAL = 12,
    /* scalar arithmetic used for the s-channel ordering bounds (Sec. 2.2.7) */
    PS_OP_ADD = 13,    /* (s|i a, s|i b) -> (s a + b)   */
    PS_OP_SUB = 14,    /* (s|i a, s|i b) -> (s a - b)   */
    PS_OP_MUL = 15,    /* (s|i a, s|i b) -> (s a b)     */
    PS_OP_DIV = 16,    /* (s|i a, s|i b) -> (s a / b)   */
    PS_OP_SQRT = 17,   /* (s a) -> (s sqrt(a))          */
    PS_OP_SQUARE = 18, /* (s a) -> (s a^2)              */
    PS_OP_MAX = 19,    /* (s|i a, s|i b) -> (s max(a,b)) */
    PS_OP_MOM_ADD = 20, /* (p a, p b) -> (p a + b)      */
    PS_OP_MOM_SUB = 21, /* (p a, p b) -> (p a - b)      */
    /* synthetic parton density (x^alpha (1-x)^beta): (s x, i alpha, i beta [, s log x]) -> (s f);
     * a given log x replaces the logarithm of x.  Pair form (s x1, i alpha, i beta, s log x1,
     * s x2, s log x2) -> (s f(x1) f(x2)), with (x1 x2)^alpha = exp(alpha (log x1 + log x2)): one
     * exponential for the two densities of a hadronic event. */
    PS_OP_PDF_POWER = 22,
    /* propagator denominator 1/((s - M^2)^2 + M^2 Gamma^2): (s s, i M, i Gamma) -> (s P). */
    PS_OP_PROPAGATOR = 23,
    /* 1 + cos^2(theta) of a momentum w.r.t. the z axis: (p q) -> (s f). */
    PS_OP_ONE_PLUS_COS2 = 24,
    /* SDE channel weight of another channel (Sec. 2.1, products of propagator denominators),
     * from momenta: (i k, p p_a, p q_1, ..., p q_k, then for each propagator four immediates
     * i kind, i mask, i M, i Gamma) -> (s P).  kind 0: s = (sum_{i in mask} q_i)^2, factor
     * 1/((s-M^2)^2 + M^2 Gamma^2); kind 1: t = (p_a - sum_{i in mask} q_i)^2, factor 1/(t-M^2)^2.
     * Bit i of mask (0-based) selects q_{i+1}. */
    PS_OP_CHANNEL_WEIGHT = 25,
    PS_OP_COUNT_ = 26
};

/* Create an empty graph with `n_random` inputs: ids 0 .. n_random-1 are the scalar
 * components of the input %0 : float[batch, n_random] (the paper's unstack). */
int ps_graph_create(int n_random, ps_graph* out);

/* Append one instruction.  out_ids receives the ids of the n_out new values (SSA:
 * ids are never redefined).  Returns PS_ERR_GRAPH for an unknown opcode, a wrong
 * number or type of arguments, or an undefined id. */
int ps_graph_add(ps_graph g, int opcode, const ps_arg* args, int n_args, int* out_ids, int n_out);

/* Output roles. */
#define PS_ROLE_MOMENTUM 0 /* momentum outputs, in order (event record [p_a, p_b, p_1..p_n]) */
#define PS_ROLE_X1 1
#define PS_ROLE_X2 2
#define PS_ROLE_WEIGHT 3
#define PS_ROLE_ALPHA 4

/* Declare the outputs: ids[k] with role roles[k].  Exactly one WEIGHT is required. */
int ps_graph_set_outputs(ps_graph g, const int* ids, const int* roles, int n);

/* Number of instructions / values / random inputs of a graph. */
int ps_graph_info(ps_graph g, int* n_instructions, int* n_values, int* n_random);

/* Text listing of the graph in the style of the paper's example (Fig. compute_graph).
 * Writes at most cap bytes (NUL-terminated) into buf; *needed receives the full size. */
int ps_graph_dump(ps_graph g, char* buf, size_t cap, size_t* needed);

int ps_graph_free(ps_graph g);

/* ----------------------------------------------------- topology builder */
/* A channel topology (Sec. 2.2, Eq. ps_decomposition) from which the builder emits the
 * instruction list: s-channel invariants in a given order with recursive bounds
 * (Sec. 2.2.7), an inward t-channel chain (Sec. 2.2.8), two-body decays, the PDF
 * convolution and beam boost, the Jacobian product, an integrand and cut_unphysical. */
#define PS_MAX_NODES 32
#define PS_MAX_LEGS 10
#define PS_NODE_LEAF 0   /* final-state particle                       */
#define PS_NODE_DECAY 1  /* s-channel 1 -> 2 node (the root: shat)      */
#define PS_NODE_TCHAIN 2 /* the root as a t-channel chain of legs       */

#define PS_INTEGRAND_NONE 0          /* f = 1                                          */
#define PS_INTEGRAND_ONE_PLUS_COS2 1 /* f = 1 + cos^2 theta of final-state particle 1  */
#define PS_INTEGRAND_PDF_PROPS 2     /* f = f(x1) f(x2) prod(resonant s-propagators)   */
#define PS_INTEGRAND_PDF_SDE 3       /* f = f(x1) f(x2) sum_c P_c, w = w_ps f alpha_c  */

typedef struct {
    int32_t kind;                 /* PS_NODE_*                                         */
    int32_t n_children;
    int32_t children[PS_MAX_LEGS];/* node ids; t-chain legs ordered from leg A to leg B */
    int32_t leaf_index;           /* leaf: final-state index 0..n-1                    */
    int32_t in_sde;               /* decay: propagator enters the SDE product           */
    double mass;                  /* leaf: on-shell mass                               */
    double prop_mass, prop_width; /* decay: Breit-Wigner if width > 0                  */
    double nu;                    /* decay with width 0: power-law exponent            */
} ps_node_desc;

typedef struct {
    int32_t n_out;       /* final-state multiplicity n                                  */
    int32_t hadronic;    /* 1: shat map, r_to_x1x2 and boost_beam; 0: fixed sqrt_s      */
    int32_t lab_frame;   /* hadronic: 1 = boost to the lab, 0 = stay in the parton frame */
    int32_t integrand;   /* PS_INTEGRAND_*                                              */
    int32_t n_nodes;     /* node 0 is the root                                          */
    int32_t n_sorder;
    int32_t sorder[PS_MAX_NODES]; /* decay nodes (not the root) in sampling order        */
    int32_t tside[PS_MAX_LEGS];   /* t-chain step i = 1..kappa-1 in tside[i]: 0 = A, 1 = B */
    int32_t vegas_dims, vegas_bins;
    double sqrt_s;       /* fixed energy                                                */
    double s_beam;       /* hadronic S                                                  */
    double a_shift;      /* auxiliary m^2 = -a for massless maps                         */
    double shat_mass, shat_width, shat_nu;
    double t_nu, ts_nu;  /* |t| map exponent; exponent of the t-chain invariants         */
    double t_prop_mass;  /* t-channel propagator mass in the SDE product                 */
    double pdf_alpha, pdf_beta;
    ps_node_desc nodes[PS_MAX_NODES];
} ps_channel_desc;

/* Random dimension count of a channel: 3n-2 (hadronic) or 3n-4. */
int ps_channel_dims(const ps_channel_desc* ch, int* n_random);

/* Build the graph of channel `which` of the set ch[0..n_ch-1] (the whole set is needed
 * for PS_INTEGRAND_PDF_SDE, whose alpha_c uses every channel's propagators).
 * Dimension order (generalising Fig. compute_graph): shat, the s-channel invariants in
 * sampling order, the t-chain invariants, x1x2, (r_phi, r_t) per t-block, (r_phi, r_theta)
 * per decay in depth-first order; VEGAS maps the first vegas_dims of them. */
int ps_graph_build_channel(const ps_channel_desc* ch, int n_ch, int which, ps_graph* out);

/* ---------------------------------------------------------------- programs */
#define PS_PRECISION_F64 0   /* every step in binary64 */
#define PS_PRECISION_MIXED 1 /* bulk kinematics in binary32, binary64 islands: invariant assembly and
                              * s - m^2, the Kallen function at threshold, the t range and small |t|,
                              * the s-order bounds and every Jacobian product; momenta, x1, x2 and
                              * alpha are written as binary32, weights as binary64 */

typedef struct {
    int32_t block_threads; /* events per tile = threads per CTA (multiple of 32, at most 256, or 512
                            * for a compiled program, PS_PROGRAM_JIT; 0 = default 128)         */
    int32_t ctas_per_sm;   /* resident CTAs requested per SM (0 = as many as fit, up to 4; a
                            * compiled program, PS_PROGRAM_JIT, caps its registers so that this
                            * many fit, and takes as many as fit when 0)                        */
    int32_t precision;     /* PS_PRECISION_*                                                  */
    int32_t flags;         /* PS_PROGRAM_* bits                                               */
} ps_options;

/* Compile the program's instruction lists into one kernel at creation (NVRTC, sm_103a): the
 * slot file in registers, the byte-code's slots and immediates as constants.  Same results as
 * the interpreter up to the rounding of fused multiply-adds across op boundaries.  Programs of
 * more than six channels are compiled one unit per channel, in parallel on host threads, and
 * linked (nvJitLink) into one kernel.  Creation fails (PS_ERR_GRAPH with the compiler's message,
 * PS_ERR_CUDA) if the kernel cannot be built.  Compiled kernels (and the split form's channel
 * units) are cached per device and source for the life of the process: a second program with
 * the same channels and options costs no compilation, and the cached modules are never unloaded. */
#define PS_PROGRAM_JIT 1

/* Generate and compile (NVRTC, no device needed) the kernel a program with these graphs and
 * options would use under PS_PROGRAM_JIT; the compiler log goes to log[log_bytes].
 * Diagnostics, read from the environment at each compilation: PS_JIT_DUMP=<file> writes the
 * generated source (the split form's units joined); PS_JIT_PTXAS_VERBOSE=1 puts the register
 * and spill report into the log; PS_JIT_SPLIT=1 or 0 forces or forbids the split form. */
int ps_jit_check(const ps_graph* graphs, int n_ch, const ps_options* opt, char* log, size_t log_bytes);

/* Compile n_ch graphs (channel c = graphs[c]) for `device`.  Every channel must declare
 * the same outputs.  Allocates the program's device constants on that device. */
int ps_program_create(const ps_graph* graphs, int n_ch, const ps_options* opt, int device, ps_program* out);

/* Upload a VEGAS grid for channel ch: edges_host[dims][bins+1], each row increasing from 0 to 1. */
int ps_program_set_vegas(ps_program p, int ch, int dims, int bins, const double* edges_host);
int ps_program_get_vegas(ps_program p, int ch, int dims, int bins, double* edges_host);

/* Output buffers (caller-owned, 16-byte aligned, in memory the device can write: device memory,
 * or pinned host memory, which the kernel then fills directly -- on a Grace-Blackwell node over
 * NVLink-C2C, with no copy; the statistics still need the device workspace).  The writes are
 * complete when the call's work on `stream` is.  Event e of channel c is stored at
 * column off_c + e, off_c = sum of the event counts of channels < c.  Momentum k, component
 * mu lives at momenta[(4k + mu) * ld + column].  momenta, x1, x2 and alpha hold double for a
 * PS_PRECISION_F64 program and float for a PS_PRECISION_MIXED program; weight is always double.
 * Pointers for roles a graph does not have may be NULL; so may any output the caller does not
 * want (it is then not written). */
typedef struct {
    void* momenta;
    void* x1;
    void* x2;
    double* weight;
    void* alpha;
    int64_t ld; /* leading dimension of momenta, in elements (>= total events) */
} ps_out_buffers;

/* Scratch memory needed by ps_generate / ps_map for these event counts (bytes). */
int ps_workspace_size(ps_program p, const int64_t* events_per_ch, size_t* bytes);

/* Generate events_per_ch[c] events of every channel in one launch, random numbers drawn
 * in-kernel by Philox4x32-10 with key = seed and counter = (event_lo, event_hi, channel,
 * dimension/2), event = event_offset + index within the channel.  Asynchronous on `stream`;
 * no allocation and no host synchronisation.  workspace: caller-owned device scratch of at
 * least ps_workspace_size bytes (256-byte aligned).  Per-channel statistics of this call are
 * kept in the program (ps_stats). */
int ps_generate(ps_program p, const int64_t* events_per_ch, uint64_t seed, uint64_t event_offset,
                const ps_out_buffers* out, void* workspace, size_t workspace_bytes, void* stream);

/* Allocation-free form of ps_generate (the paper has no counterpart): the same generation,
 * with the per-tile scratch taken from a fixed array that the library keeps in device memory
 * (131072 tiles of block_threads events each -- 16,777,216 events per call at the default block
 * of 128 -- 4 MiB held on every device that loads the library, until the process exits).  For
 * callers that cannot call cudaMalloc or hand out device memory: code running inside a host
 * framework that owns every device allocation, or a loop that must not let an allocation
 * synchronise the device.  The call allocates nothing.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *    that device current; make that first call before any stream capture.
 *  - Event counts needing more tiles than the array holds are rejected with PS_ERR_CAPACITY.
 *  - All calls share the one array, which keeps the last call's contents; every tile record is
 *    written before it is read, so nothing needs clearing.  Calls whose kernels overlap on the
 *    GPU (different streams, or different threads, without ordering) race on it: order them. */
int ps_generate_noalloc(ps_program p, const int64_t* events_per_ch, uint64_t seed, uint64_t event_offset,
                        const ps_out_buffers* out, void* stream);

/* Explicit-input form: map `batch` given points r_dev[j * ld_r + e] (SoA, j < n_random) of
 * channel ch.  Outputs start at column 0. */
int ps_map(ps_program p, int ch, int64_t batch, const double* r_dev, int64_t ld_r,
           const ps_out_buffers* out, void* workspace, size_t workspace_bytes, void* stream);

/* CUDA-graph executor of ps_generate.  ps_exec_create captures one ps_generate call (the map
 * kernel and the reduction) for fixed event counts, output buffers and workspace into a CUDA
 * graph and instantiates it; ps_exec_launch replays it on `stream` with a new seed and event
 * offset, which it writes into the captured kernel nodes, so that successive replays draw new
 * events without a new capture.  The buffers given at creation must stay valid while the
 * executor is used.  Capture happens on a private stream of the program's device.  A compiled
 * program's kernel (PS_PROGRAM_JIT) is captured and updated through the CUDA driver API, since
 * it comes from a module loaded at run time; the behaviour is the same. */
typedef struct ps_exec_s* ps_exec;
int ps_exec_create(ps_program p, const int64_t* events_per_ch, const ps_out_buffers* out, void* workspace,
                   size_t workspace_bytes, ps_exec* exec_out);
int ps_exec_launch(ps_exec e, uint64_t seed, uint64_t event_offset, void* stream);
int ps_exec_free(ps_exec e);

typedef struct {
    double n;          /* events                */
    double n_nonzero;  /* events with w != 0    */
    double sum_w;
    double sum_w2;
    double max_w;
} ps_channel_stats;

/* Copy the statistics of the last ps_generate / ps_map (synchronises `stream`; the copy is a
 * one-block kernel into host-mapped memory, so it does not wait for copy-engine traffic); in
 * streaming mode (ps_stats_accumulate) the running statistics of every launch since the
 * mode was enabled. */
int ps_stats(ps_program p, ps_channel_stats* host_out, int n_ch, void* stream);

/* Streaming mode for event samples generated in chunks (the integral over all chunks,
 * Sec. 2 Monte Carlo estimate from the per-channel sums).  enable != 0 zeroes the program's
 * statistics and makes every later reduction, including those of captured ps_exec graphs,
 * add its per-channel sums to them (n, n_nonzero, sum_w, sum_w2; max_w by maximum) in stream
 * order, so a stream of chunks needs one ps_stats read at its end.  enable == 0 restores
 * per-launch statistics.  Enqueued on `stream` (asynchronous); the mode applies to launches
 * ordered after it.  Errors: PS_ERR_INVALID_ARGUMENT for a null program, PS_ERR_CUDA. */
int ps_stats_accumulate(ps_program p, int enable, void* stream);

/* VEGAS training (the adaptive sampling of Sec. 3.2.2, Lepage's grid refinement): while
 * enabled, ps_generate, ps_map and executors also accumulate, per channel, mapped dimension j
 * and bin k, the sum of w^2 over events whose r_j falls in bin k.  Two extra kernels per launch
 * read the stored weights (the weight output is then required, else PS_ERR_INVALID_ARGUMENT) and
 * add the sums in a fixed order: 128 equal slices of each channel's events, each summed in
 * event order, then the slices in order.  The histogram, and every grid adapted from it, is
 * therefore the same bit for bit for the same events, whatever the block size, CTA count or
 * compiled form.  The first enable allocates the partial sums (n_channels x 128 x dims x bins
 * doubles); PS_ERR_CAPACITY if dims > 64, bins > 256 or dims x bins > 4096. */
int ps_vegas_training(ps_program p, int enable);
/* Copy channel ch's accumulated histogram [dims][bins] (synchronises). */
int ps_vegas_histogram(ps_program p, int ch, double* hist_host, void* stream);
/* Rebin channel ch from its histogram (Lepage: 3-point smoothing, compression exponent
 * alpha), upload the new grid and clear the histogram (synchronises). */
int ps_vegas_adapt(ps_program p, int ch, double alpha, void* stream);

/* Device status counters of the program since the last reset: [0] non-finite weights
 * before the cut, [1] events cut by cut_unphysical, [2] grid index clamps.  Synchronises. */
int ps_status(ps_program p, int64_t* counters_host, int n, void* stream);
int ps_status_reset(ps_program p, void* stream);

int ps_program_free(ps_program p);

/* ------------------------------------------------------------------------------------------
 * Learned proposal: rational-quadratic-spline coupling flow (neural importance sampling with
 * rational-quadratic spline transformations, Sec. 3.2.2; spline of Durkan et al. 2019, whose
 * single-bin case is the RQF of Sec. 2.3).  The flow maps z in (0,1)^d, drawn from Philox,
 * to r in (0,1)^d, which feeds ps_map's explicit-input mode; the event weight becomes
 * w = w_map |dr/dz|  (the flow density in r is |dz/dr|).
 *
 * Coupling layer l transforms the dims whose index has bit (l mod nbits) different from
 * ((l div nbits) mod 2), nbits = ceil(log2 d), for d <= 16, and the dims j with
 * j mod 3 == l mod 3 for 16 < d <= 24 (at most 8 transformed and 16 conditioning dims, the
 * shape of the fused tensor-core layer), conditioned on the other dims through the MLP
 *     A -> Linear(hidden) -> SiLU -> Linear(hidden) -> SiLU -> Linear(n_B (3 bins + 1)),
 * giving per transformed dim `bins` width logits, `bins` height logits and bins+1 derivative
 * pre-activations:  widths/heights = 1e-3 + (1 - bins 1e-3) softmax(.), knot derivatives =
 * 1e-3 + softplus(.).  The GEMMs run on tensor cores with bfloat16 operands and FP32
 * accumulation; splines, log-determinants and the backward pass run in FP32.
 *
 * Parameters (logical layout of get/set/gradients, float32, per layer l in order):
 *     W1 [hidden][n_A], b1 [hidden], W2 [hidden][hidden], b2 [hidden],
 *     W3 [n_B (3 bins + 1)][hidden], b3 [n_B (3 bins + 1)]
 * (rows of W3/b3: transformed dim q in ps_flow_mask order, then widths, heights,
 * derivatives).  A new flow starts at the identity: W3 = 0 and derivative biases
 * log(expm1(1 - 1e-3)); hidden weights uniform in +-1/sqrt(fan_in) from `init_seed`.
 *
 * Training minimises the importance-weighted forward KL divergence, on the last sampled
 * batch:  L = - sum_b (w_b / sum w) log g(r_b),  w_b = w_map_b |dr/dz|_b, with w_b held fixed
 * (its gradient is not taken), by Adam (beta 0.9, 0.999, eps 1e-8).
 * ------------------------------------------------------------------------------------------ */
typedef struct ps_flow_s* ps_flow;

/* Message of the last failed flow call on this thread. */
const char* ps_flow_last_error(void);

/* Create a flow on `device`: 2 <= dims <= 24, 1 <= n_layers <= 8, 1 <= bins <= 32,
 * hidden a multiple of 16 in [16, 512], 1 <= max_batch <= 2^24 events per sample chunk.
 * Allocates the parameters, Adam state and the activations of max_batch events
 * (about (L (10 hidden + 4 P) + 4 P + 20 hidden) bytes per event).  Synchronises. */
int ps_flow_create(int dims, int n_layers, int bins, int hidden, int64_t max_batch, uint64_t init_seed, int device,
                   ps_flow* out);
int ps_flow_free(ps_flow f);
/* Shape and the number of logical parameters. Any output pointer may be null. */
int ps_flow_info(ps_flow f, int* dims, int* n_layers, int* bins, int* hidden, int64_t* n_params);
/* Transformed dims of `layer` (ascending) into transformed[<= dims]. */
int ps_flow_mask(ps_flow f, int layer, int* transformed, int* n_transformed);
/* Copy the FP32 master parameters to/from host memory in the logical layout (n must equal
 * n_params).  Synchronous. */
int ps_flow_get_params(ps_flow f, float* host, int64_t n);
int ps_flow_set_params(ps_flow f, const float* host, int64_t n);

/* Draw `batch` events on `stream`: z from Philox4x32-10 with counter (event lo, event hi,
 * 0x466C6F77, j/2) and key (seed lo, seed hi), dims 2i and 2i+1 from words 0 and 1 of the
 * block i, z = (top 23 bits + 1/2) 2^-23; then r = flow(z), clamped to [1e-7, 1 - 1e-7].
 * Device outputs (SoA, column = event, leading dimension ld_r >= batch):
 *     r[j ld_r + b] (double, required), logdet[b] = log |dr/dz| (double, may be null),
 *     z[j ld_r + b] (double, may be null).
 * Batches above max_batch run in chunks; a later ps_flow_train_step needs batch <= max_batch
 * (it uses the activations of this call).  Asynchronous. */
int ps_flow_sample(ps_flow f, int64_t batch, uint64_t seed, uint64_t event_offset, double* r, int64_t ld_r,
                   double* logdet, double* z, void* stream);
/* Sampling for inference (no training step can follow): the same draws and outputs as
 * ps_flow_sample, any batch size.  With hidden = 128, bins <= 18 and at most 8 transformed dims
 * per layer, each layer runs as one fused kernel (the three GEMMs, then the splines; weights in
 * shared memory): with 16 bins on the tcgen05 tensor cores (FP32 accumulators in TMEM, one event
 * per TMEM lane), otherwise with warp-level MMAs and the hidden activations in registers.  Other
 * shapes run layer by layer.
 * Allocates its 2^20-event working buffers on first use.  Asynchronous. */
int ps_flow_generate(ps_flow f, int64_t batch, uint64_t seed, uint64_t event_offset, double* r, int64_t ld_r,
                     double* logdet, double* z, void* stream);
/* The inverse map: z = flow^-1(r) and logq[b] = log g(r_b) = -log |dr/dz| for `batch` points r
 * (device, SoA [dims][ld_r], double); z has the layout of r; logq may be null.  Uses the fused
 * layer kernels where ps_flow_generate does (leaving the activations of the last sample intact);
 * otherwise runs layer by layer in chunks of max_batch and discards those activations.
 * Asynchronous. */
int ps_flow_inverse(ps_flow f, int64_t batch, const double* r, int64_t ld_r, double* z, double* logq,
                    void* stream);
/* w[b] = w_map[b] exp(logdet[b]) (non-finite -> 0); device pointers.  Asynchronous. */
int ps_flow_weights(ps_flow f, int64_t batch, const double* w_map, const double* logdet, double* w, void* stream);
/* One Adam step with learning rate lr on the loss of the last sampled batch, whose phase-space
 * weights w_map (device, [batch]) the caller computed from that batch's r.  Asynchronous. */
int ps_flow_train_step(ps_flow f, const double* w_map, double lr, void* stream);
/* The loss gradient of the last sampled batch in the logical layout (host, n = n_params) and
 * the loss value, without updating parameters.  Synchronises `stream`. */
int ps_flow_gradients(ps_flow f, const double* w_map, float* host, int64_t n, double* loss, void* stream);
/* Number of tensor-core completion waits of the fused sampling kernels that ran out since the
 * last call (the count is cleared).  Each wait is bounded; a timeout leaves that tile's outputs
 * invalid, and the kernel still drains its MMAs and frees its TMEM before it returns, so the
 * context stays usable.  0 in a healthy run.  Synchronises the device. */
int ps_flow_status(ps_flow f, int64_t* timeouts);
/* Bound of every completion wait of the fused sampling kernels, in polls of the mbarrier
 * (default 2^24; polls <= 0 restores it).  A small bound makes the waits run out: the failure
 * path of ps_flow_status can be exercised without faulting or hanging the device. */
int ps_flow_set_wait_limit(ps_flow f, int polls);
/* Test flags of the fused tcgen05 kernels (0 = none, the default).  Bit 0: each group of a CTA
 * withholds the completion signal of its first MMA chain, so that the bounded wait on it runs
 * out (use with a small ps_flow_set_wait_limit); the outputs of that run are invalid, the
 * timeouts appear in ps_flow_status, and nothing faults or hangs.  Bit 1: ps_flow_sample (the
 * training forward) runs layer by layer -- separate GEMM, gather and spline kernels -- instead
 * of the tcgen05 layer kernel, so that the two forms can be compared.  Tests only. */
int ps_flow_set_debug(ps_flow f, int flags);
/* Loss and sum of w of the last train_step / gradients call.  Synchronises `stream`. */
int ps_flow_loss(ps_flow f, double* loss, double* sum_w, void* stream);

/* ------------------------------------------------------------------------------------------
 * Inverse maps and global multichannel weights.
 *
 * Every mapping of the phase-space construction is invertible (Sec. 2), and the global
 * multichannel method (Kleiss and Pittau; Eq. channel_densities and Eq. multi-channel-standard)
 * weights an event x by w = f(x) / g(x) with g = sum_i alpha_i g_i, where g_i(x) =
 * |d G_i^-1(x) / dx| is channel i's density at x.  g_i is 1/J_i(r_i), J_i the phase-space
 * weight of channel i (integrand "none") at r_i = G_i^-1(x): the inverse below gives r_i, a
 * program of the channels with integrand "none" gives J_i through ps_map, and
 * ps_global_weights combines them.
 * ------------------------------------------------------------------------------------------ */

/* r = G^-1(x) of program channel `ch` for `batch` events, in FP64 on the device:
 *   momenta  [4 (n+2)][ld_m] lab-frame event records [p_a, p_b, p_1..p_n] (row 4 i + mu), as
 *            written by ps_generate / ps_map;  x1, x2 [batch] (hadronic channels; else null);
 *   r        [n_random][ld_r] output, the random numbers the forward map takes to these momenta
 *            (VEGAS inverted with the program's current grid);
 *   P        [batch] output or null: the channel's SDE weight prod 1/|q^2 - M^2 + i M G|^2 of its
 *            s-channel propagators in the SDE list and t-channel propagators, from the momenta.
 * `desc` must describe program channel `ch` (same dimension count and VEGAS dimensions).
 * Invariants come from the leaves in a collinear-safe form; the beam boost is undone on the
 * light cone.  Asynchronous. */
int ps_inverse_map(ps_program p, int ch, const ps_channel_desc* desc, int64_t batch, const double* momenta,
                   int64_t ld_m, const double* x1, const double* x2, double* r, int64_t ld_r, double* P,
                   void* stream);

/* Global multichannel weights (device arrays):  w[b] = f_b / sum_j alpha[j] / J[j ld_j + b]
 * (terms with J <= 0 contribute no density; w = 0 if none is left), where f_b = f[b] if f is
 * given, else  pdf(x1) pdf(x2) sum_j P[j ld_p + b]  with pdf(x) = x^pdf_alpha (1-x)^pdf_beta
 * (x1 = x2 = null: the PDF factor is 1).  alpha: host array of n_ch non-negative channel
 * weights (normally summing to 1).  Asynchronous. */
int ps_global_weights(int n_ch, int64_t batch, const double* J, int64_t ld_j, const double* P, int64_t ld_p,
                      const double* alpha, const double* x1, const double* x2, double pdf_alpha, double pdf_beta,
                      const double* f, double* w, void* stream);

/* ------------------------------------------------------------------------------------------
 * Unweighting (Sec. "Unweighting and file output"): the maximum weight is estimated allowing a
 * given amount of over-weight events relative to the total cross section (0.1% in the paper's
 * validation runs), and events are accepted against it.
 *
 *   w_max(eps) = the smallest t >= 0 with  sum_b max(0, w_b - t) <= eps * sum_b w_b
 *
 * (the share of the cross section above w_max is at most eps).  Event b is accepted iff
 * u_b w_max < w_b, with u_b the first uniform of the generator's Philox point of event
 * (event_offset + b) in stream 0x556E7700 (counter (event lo, event hi, 0x556E7700, 0), key
 * (seed lo, seed hi), top 52 bits of words 1:0, (k + 1/2) 2^-52); an accepted event keeps the
 * weight max(w_b, w_max), so the accepted weights estimate sum_b w_b without bias.
 * Weights that are negative or not finite are counted and skipped (never accepted).
 * All pointers are device pointers; the calls are asynchronous on `stream` and reproducible
 * bit for bit for a given n.
 * ------------------------------------------------------------------------------------------ */
const char* ps_unweight_last_error(void);
/* Bytes of workspace for n weights (the workspace must be 256-byte aligned). */
int ps_unweight_workspace_size(int64_t n, size_t* bytes);
/* result[5] (device doubles) <- { w_max, sum of valid w, max w, number of weights above w_max
 * (the over-weight events), number of invalid weights }.  eps >= 0. */
int ps_unweight_max(const double* w, int64_t n, double eps, double* result, void* workspace, size_t ws_bytes,
                    void* stream);
/* Accept against *w_max (device scalar, e.g. result[0] above): the indices of the accepted
 * events in increasing order into idx[], their weights max(w, w_max) into w_out[] (both with
 * room for n), and their number into *n_accepted (device int64). */
int ps_unweight_select(const double* w, int64_t n, const double* w_max, uint64_t seed, uint64_t event_offset,
                       int64_t* idx, double* w_out, int64_t* n_accepted, void* workspace, size_t ws_bytes,
                       void* stream);

/* Number of kernel launches issued by the library since load (all programs). */
int64_t ps_launch_count(void);

/* ------------------------------------------------------------------------------------------
 * FP64-pipe probes (no counterpart in the paper: they measure the device the FP64 kernels'
 * roofline is stated against).  ps_fp64_probe launches `blocks` CTAs of 256 threads on
 * `stream`; every thread runs `iters` iterations and writes one double to sink[] (device,
 * blocks x 256 doubles, caller-owned).  Asynchronous; the caller times it with CUDA events.
 *   PS_PROBE_DFMA/DADD/DMUL: eight independent chains of that instruction per iteration, i.e.
 *     8 x iters x blocks x 256 FP64 instructions per launch (the issue rate's numerator);
 *   PS_PROBE_EMPTY and the function kinds: one call of the function per iteration (sincospi:
 *     one call, both results) with arguments spread over a fixed range, next to the empty loop;
 *     the difference of their FP64-pipe instruction counters (a profiler's) over blocks x 256 x
 *     iters is the function's FP64-pipe instructions per call.
 * Returns PS_ERR_INVALID_ARGUMENT for an unknown kind, blocks < 1, iters < 1 or a null sink. */
#define PS_PROBE_DFMA 0
#define PS_PROBE_DADD 1
#define PS_PROBE_DMUL 2
#define PS_PROBE_EMPTY 9
#define PS_PROBE_DIV 10
#define PS_PROBE_SQRT 11
#define PS_PROBE_RSQRT 12
#define PS_PROBE_EXP 13
#define PS_PROBE_EXPM1 14
#define PS_PROBE_LOG 15
#define PS_PROBE_LOG1P 16
#define PS_PROBE_POW 17
#define PS_PROBE_ATAN 18
#define PS_PROBE_ATAN2 19
#define PS_PROBE_TAN 20
#define PS_PROBE_SIN 21
#define PS_PROBE_COS 22
#define PS_PROBE_SINCOSPI 23
int ps_fp64_probe(int kind, int blocks, int iters, double* sink, void* stream);

/* ------------------------------------------------------------------------------------------
 * The device helpers of the mixed-precision form at the edges of its FP64 islands (no
 * counterpart in the paper), exposed so that their results can be checked against the
 * hardware's conversions and FP64 functions.  ps_mixed_helpers applies helper `kind` to each of
 * the n values of in[] and writes out[] (both device, caller-owned; in[] and out[] of the types
 * below), asynchronously on `stream`:
 *   PS_MIXED_F2D     float  -> double: IEEE 754 widening (exact), on the integer ALU;
 *   PS_MIXED_D2F     double -> float: IEEE 754 narrowing, round to nearest even, integer ALU;
 *   PS_MIXED_SQRT64  double -> double: sqrt(x) from a seed (exponent on the integer ALU, fraction
 *                    from a float instruction) and one FP64 Newton step, relative error below
 *                    1e-13 for normal x > 0; 0 for x <= 0 or NaN;
 *   PS_MIXED_RCP64   double -> double: 1/x the same way, for normal x of either sign;
 *   PS_MIXED_SINCOS_TURN  double r -> the doubles cos(2 pi r), sin(2 pi r) at out[2i], out[2i+1]:
 *                    the FP64 kernels' azimuth (a table of 256 points and short Taylor series);
 *   PS_MIXED_TAN_QUARTER  double x -> double tan(x) for |x| <= pi/4: the FP64 Breit-Wigner map's
 *                    tangent (a double-double table of 129 points and a short Taylor series).
 * Returns PS_ERR_INVALID_ARGUMENT for an unknown kind, n < 0, or a null pointer with n > 0. */
#define PS_MIXED_F2D 0
#define PS_MIXED_D2F 1
#define PS_MIXED_SQRT64 2
#define PS_MIXED_RCP64 3
#define PS_MIXED_SINCOS_TURN 4
#define PS_MIXED_TAN_QUARTER 5
int ps_mixed_helpers(int kind, const void* in, void* out, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PS_H */
