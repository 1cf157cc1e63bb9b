/* Operation counter for the FP64 oracle -- TEST AND MEASUREMENT INFRASTRUCTURE ONLY.
 *
 * Force-included (g++ -include, the oracle compiled as C++) ahead of ps_oracle.c to build a
 * third copy of the oracle, liboracle_count.so, in which every `double` is a counting double:
 * a one-member class that performs the same IEEE operation and adds one to the counter of its
 * class.  The classes are add (also subtract), mul, div, sqrt, one per elementary function
 * (exp, expm1, log, log1p, pow, atan, atan2, tan, sin, cos), cmp (comparisons) and other
 * (fabs, fmin, fmax, floor).  The copy is built with ORC_BOOKKEEPING = 0, so the condition
 * numbers that the parity tests read are not computed and not counted: what remains is the
 * method's own arithmetic, step by step in the paper's order.  Counts are per process (no
 * OpenMP in this copy); orc_count_reset() and orc_count_get() read them.
 *
 * The class keeps the layout of a double (sizeof 8, standard layout), so the oracle's arrays and
 * its batch entry points keep their binary interface.
 */
#ifndef ORC_OP_COUNT_H
#define ORC_OP_COUNT_H
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>

enum {
    ORC_C_ADD, ORC_C_MUL, ORC_C_DIV, ORC_C_SQRT, ORC_C_EXP, ORC_C_EXPM1, ORC_C_LOG, ORC_C_LOG1P,
    ORC_C_POW, ORC_C_ATAN, ORC_C_ATAN2, ORC_C_TAN, ORC_C_SIN, ORC_C_COS, ORC_C_CMP, ORC_C_OTHER,
    ORC_C_N
};

static unsigned long long orc_counts[ORC_C_N];

extern "C" void orc_count_reset(void) { memset(orc_counts, 0, sizeof orc_counts); }
extern "C" int orc_count_classes(void) { return ORC_C_N; }
extern "C" void orc_count_get(unsigned long long* out)
{
    for (int k = 0; k < ORC_C_N; ++k) out[k] = orc_counts[k];
}

struct orc_cd {
    double v;
    orc_cd() = default;
    constexpr orc_cd(double x) : v(x) {}
    template <class T, class = typename std::enable_if<std::is_arithmetic<T>::value>::type>
    constexpr orc_cd(T x) : v(static_cast<double>(x)) {}
    template <class T, class = typename std::enable_if<std::is_arithmetic<T>::value>::type>
    explicit operator T() const { return static_cast<T>(v); }
    orc_cd& operator+=(orc_cd o) { ++orc_counts[ORC_C_ADD]; v += o.v; return *this; }
    orc_cd& operator-=(orc_cd o) { ++orc_counts[ORC_C_ADD]; v -= o.v; return *this; }
    orc_cd& operator*=(orc_cd o) { ++orc_counts[ORC_C_MUL]; v *= o.v; return *this; }
    orc_cd& operator/=(orc_cd o) { ++orc_counts[ORC_C_DIV]; v /= o.v; return *this; }
};
static_assert(sizeof(orc_cd) == sizeof(double), "counting double must keep the layout of a double");
static_assert(std::is_standard_layout<orc_cd>::value && std::is_trivially_copyable<orc_cd>::value,
              "counting double must be a plain value");

static inline orc_cd operator+(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_ADD]; return orc_cd(a.v + b.v); }
static inline orc_cd operator-(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_ADD]; return orc_cd(a.v - b.v); }
static inline orc_cd operator*(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_MUL]; return orc_cd(a.v * b.v); }
static inline orc_cd operator/(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_DIV]; return orc_cd(a.v / b.v); }
static inline orc_cd operator-(orc_cd a) { return orc_cd(-a.v); }
static inline orc_cd operator+(orc_cd a) { return a; }
static inline bool operator<(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_CMP]; return a.v < b.v; }
static inline bool operator>(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_CMP]; return a.v > b.v; }
static inline bool operator<=(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_CMP]; return a.v <= b.v; }
static inline bool operator>=(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_CMP]; return a.v >= b.v; }
static inline bool operator==(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_CMP]; return a.v == b.v; }
static inline bool operator!=(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_CMP]; return a.v != b.v; }

#define ORC_CD_FN1(name, cls)                                                           \
    static inline orc_cd name(orc_cd a) { ++orc_counts[cls]; return orc_cd(::name(a.v)); }
ORC_CD_FN1(sqrt, ORC_C_SQRT)
ORC_CD_FN1(exp, ORC_C_EXP)
ORC_CD_FN1(expm1, ORC_C_EXPM1)
ORC_CD_FN1(log, ORC_C_LOG)
ORC_CD_FN1(log1p, ORC_C_LOG1P)
ORC_CD_FN1(atan, ORC_C_ATAN)
ORC_CD_FN1(tan, ORC_C_TAN)
ORC_CD_FN1(sin, ORC_C_SIN)
ORC_CD_FN1(cos, ORC_C_COS)
ORC_CD_FN1(fabs, ORC_C_OTHER)
ORC_CD_FN1(floor, ORC_C_OTHER)
#undef ORC_CD_FN1
static inline orc_cd pow(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_POW]; return orc_cd(::pow(a.v, b.v)); }
static inline orc_cd atan2(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_ATAN2]; return orc_cd(::atan2(a.v, b.v)); }
static inline orc_cd fmin(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_OTHER]; return orc_cd(::fmin(a.v, b.v)); }
static inline orc_cd fmax(orc_cd a, orc_cd b) { ++orc_counts[ORC_C_OTHER]; return orc_cd(::fmax(a.v, b.v)); }
static inline bool isfinite(orc_cd a) { return std::isfinite(a.v); }

#define double orc_cd
#endif
