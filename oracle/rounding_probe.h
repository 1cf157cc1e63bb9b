/* Rounding probe for the FP64 oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Force-included (gcc -include) ahead of ps_oracle.c to build a second copy of the oracle,
 * liboracle_rounding.so, whose elementary functions (exp, expm1, log, log1p, pow, atan, atan2,
 * tan, sin, cos) return their libm result moved by a random whole number of ulps in [-2, 2].
 * Basic arithmetic and sqrt are correctly rounded on every IEEE machine and stay untouched.
 *
 * Two correct FP64 evaluations of the same formulas differ mostly in these functions: libm
 * implementations are accurate to 1-2 ulps, not correctly rounded, and the differences are
 * amplified by the map wherever it is ill-conditioned (sliver ranges, thresholds, near-backward
 * scattering), compounded through nested invariants.  Re-running the oracle with random
 * perturbations of that size and taking the spread of the results is the stochastic-arithmetic
 * estimate of its rounding sensitivity (Vignes' CESTAC method: the spread of several runs
 * with randomly perturbed roundings estimates the number of exact digits of a result).  The
 * parity tests use the spread as a per-event tolerance next to the analytic condition numbers.
 *
 * The perturbation stream is a 64-bit xorshift, reset by orc_rounding_seed(); the copy is built
 * without OpenMP so that one seed gives one deterministic sequence of perturbations.
 */
#ifndef ORC_ROUNDING_PROBE_H
#define ORC_ROUNDING_PROBE_H
#include <math.h>
#include <stdint.h>

static uint64_t orc_rounding_state = 1;

void orc_rounding_seed(uint64_t seed)
{
    orc_rounding_state = seed * 0x9E3779B97F4A7C15ull | 1ull;
}

static inline double orc_rounding_move(double v)
{
    uint64_t s = orc_rounding_state;
    s ^= s << 13;
    s ^= s >> 7;
    s ^= s << 17;
    orc_rounding_state = s;
    int k = (int)(s % 5u) - 2;
    for (; k > 0; --k) v = nextafter(v, INFINITY);
    for (; k < 0; ++k) v = nextafter(v, -INFINITY);
    return v;
}

static inline double orc_r_exp(double x) { return orc_rounding_move(exp(x)); }
static inline double orc_r_expm1(double x) { return orc_rounding_move(expm1(x)); }
static inline double orc_r_log(double x) { return orc_rounding_move(log(x)); }
static inline double orc_r_log1p(double x) { return orc_rounding_move(log1p(x)); }
static inline double orc_r_pow(double x, double y) { return orc_rounding_move(pow(x, y)); }
static inline double orc_r_atan(double x) { return orc_rounding_move(atan(x)); }
static inline double orc_r_atan2(double y, double x) { return orc_rounding_move(atan2(y, x)); }
static inline double orc_r_tan(double x) { return orc_rounding_move(tan(x)); }
static inline double orc_r_sin(double x) { return orc_rounding_move(sin(x)); }
static inline double orc_r_cos(double x) { return orc_rounding_move(cos(x)); }

#define exp(x) orc_r_exp(x)
#define expm1(x) orc_r_expm1(x)
#define log(x) orc_r_log(x)
#define log1p(x) orc_r_log1p(x)
#define pow(x, y) orc_r_pow(x, y)
#define atan(x) orc_r_atan(x)
#define atan2(y, x) orc_r_atan2(y, x)
#define tan(x) orc_r_tan(x)
#define sin(x) orc_r_sin(x)
#define cos(x) orc_r_cos(x)

#endif
