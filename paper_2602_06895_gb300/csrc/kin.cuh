// kin.cuh -- FP64 kinematic helpers shared by the forward interpreter (kernels.cu) and the
// inverse map (inverse.cu): four-momenta, the Kallen function, pure boosts and the t range of
// a 2->2 block.
#pragma once
#include <cmath>

namespace ps {
namespace dev {

constexpr double kPi = 3.141592653589793238462643383279502884;

// Decisions on doubles taken on their bit patterns in the integer ALU, which leaves the FP64
// pipe (1/64 of the FP32 rate) to arithmetic: IEEE doubles of one sign order like their bit
// patterns read as signed integers.
constexpr long long kInfBits = 0x7FF0000000000000LL;
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }
// isfinite(v)
__device__ __forceinline__ bool finite_bits(double v) { return (dbits(v) & kInfBits) != kInfBits; }
// 0 < v <= 1 (false for NaN)
__device__ __forceinline__ bool in_unit_bits(double v) {
    const long long b = dbits(v);
    return b > 0 && b <= 0x3FF0000000000000LL;
}
// v > 0 (false for NaN and -0)
__device__ __forceinline__ bool pos_bits(double v) {
    const long long b = dbits(v);
    return b > 0 && b <= kInfBits;
}
// a >= b for b >= +0 (false for NaN a)
__device__ __forceinline__ bool ge_pos_bits(double a, double b) {
    const long long x = dbits(a);
    return x >= dbits(b) && x <= kInfBits;
}
// v < -c and v > c for a constant c > 0 and finite v
__device__ __forceinline__ bool below_neg_bits(double v, double c) {
    const long long b = dbits(v);
    return b < 0 && (b & 0x7FFFFFFFFFFFFFFFLL) > dbits(c);
}
__device__ __forceinline__ bool above_pos_bits(double v, double c) { return dbits(v) > dbits(c); }
// an integer 0 <= v < 2^31 held in a double (byte-code immediates), decoded from its bits:
// v = 1.m 2^e gives (1m) >> (52 - e)
__device__ __forceinline__ int small_int(double v) {
    const unsigned long long b = static_cast<unsigned long long>(dbits(v));
    const int e = static_cast<int>((b >> 52) & 0x7FF) - 1023;
    if (e < 0) return 0;
    return static_cast<int>(((b & 0xFFFFFFFFFFFFFULL) | 0x10000000000000ULL) >> (52 - e));
}
// floor(y) for y >= 0 as the conversion to int gives it (saturating at 2^31 - 1; NaN and
// negative y give 0), from the bits: y = 1.m 2^e gives (1m) >> (52 - e)
__device__ __forceinline__ int floor_small(double y) {
    const long long b = dbits(y);
    const int e = static_cast<int>(b >> 52) - 1023;  // b < 0 (negative y) gives e < 0
    if (e < 0) return 0;
    if (e > 30) return b > kInfBits ? 0 : 0x7FFFFFFF;
    return static_cast<int>(((static_cast<unsigned long long>(b) & 0xFFFFFFFFFFFFFULL) | 0x10000000000000ULL) >> (52 - e));
}
// the double of an int 0 <= k < 2^31, from the bits
__device__ __forceinline__ double small_to_double(int k) {
    if (k <= 0) return 0.0;
    const int msb = 31 - __clz(k);
    const unsigned long long m = (static_cast<unsigned long long>(k) << (52 - msb)) & 0xFFFFFFFFFFFFFULL;
    return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(1023 + msb) << 52) | m));
}
// fmax(a, b) on the bit patterns: doubles order like the integers b ^ (0x7FF..F if negative);
// a NaN operand gives the other one
__device__ __forceinline__ double fmax_bits(double a, double b) {
    const long long x = dbits(a), y = dbits(b);
    const bool nan_a = (x & 0x7FFFFFFFFFFFFFFFLL) > kInfBits, nan_b = (y & 0x7FFFFFFFFFFFFFFFLL) > kInfBits;
    const long long kx = x ^ ((x >> 63) & 0x7FFFFFFFFFFFFFFFLL), ky = y ^ ((y >> 63) & 0x7FFFFFFFFFFFFFFFLL);
    return nan_a ? b : (nan_b ? a : (kx >= ky ? a : b));
}
// fmin(fmax(x, lo), hi) for 0 <= lo <= hi: NaN and values below lo give lo, +inf gives hi
__device__ __forceinline__ double clamp_nonneg(double x, double lo, double hi) {
    const long long b = dbits(x);
    if (b < dbits(lo) || b > kInfBits) return lo;
    return b > dbits(hi) ? hi : x;
}

struct P4 {
    double e, x, y, z;
};

__device__ __forceinline__ P4 p4_add(P4 a, P4 b) { return {a.e + b.e, a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ P4 p4_sub(P4 a, P4 b) { return {a.e - b.e, a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double p4_sq(P4 a) { return a.e * a.e - a.x * a.x - a.y * a.y - a.z * a.z; }

// Kallen lambda(x, y, z) = (x - y - z)^2 - 4 y z (x >= 0), without cancellation:
//   y, z >= 0: (x - (sqrt y + sqrt z)^2)(x - (sqrt y - sqrt z)^2)
//   y, z <= 0: x^2 + 2x(|y| + |z|) + (|y| - |z|)^2  (space-like legs of a t-chain)
//   mixed:     (x - y - z)^2 - 4 y z                (-4yz >= 0)
// clamped at zero.
// The branches are taken on the bit patterns (integer ALU); y = z = 0 (two massless legs) is x^2.
__device__ __forceinline__ bool zero_bits(double v) { return (dbits(v) << 1) == 0; }       // +-0
__device__ __forceinline__ bool nonneg_bits(double v) { return dbits(v) >= 0 || zero_bits(v); }
__device__ __forceinline__ bool nonpos_bits(double v) { return dbits(v) <= 0; }            // includes -0
__device__ __forceinline__ double kallen(double x, double y, double z) {
    double l;
    if (zero_bits(y) && zero_bits(z)) {
        l = x * x;
    } else if (nonneg_bits(y) && nonneg_bits(z)) {
        double ry = sqrt(y), rz = sqrt(z);
        double hi = ry + rz, lo = ry - rz;
        l = (x - hi * hi) * (x - lo * lo);
    } else if (nonpos_bits(y) && nonpos_bits(z)) {
        double d = z - y;
        l = x * x - 2.0 * x * (y + z) + d * d;
    } else {
        double d = x - y - z;
        l = d * d - 4.0 * y * z;
    }
    return pos_bits(l) ? l : 0.0;  // clamped at zero (NaN -> 0)
}
// lambda(x, m1^2, m2^2) from the masses m1, m2 >= 0 themselves: the factorised form above with
// sqrt(m^2) replaced by m.  For a double m the correctly rounded sqrt of fl(m^2) is m exactly
// (its error is below half an ulp of m), so this equals kallen(x, m1 m1, m2 m2) bit for bit,
// without the two square roots.
__device__ __forceinline__ double kallen_m(double x, double m1, double m2) {
    double l;
    if (zero_bits(m1 * m1) && zero_bits(m2 * m2)) {
        l = x * x;
    } else {
        double hi = m1 + m2, lo = m1 - m2;
        l = fma(-hi, hi, x) * fma(-lo, lo, x);  // explicit: the same roundings with constant masses
    }
    return pos_bits(l) ? l : 0.0;
}

// Pure boosts out of the rest frame of q (mass mq) sharing their reciprocals: 1/mq and
// 1/(mq (E_q + mq)) are taken once per frame, for every momentum boosted with it.
struct BoostFrame {
    double e, x, y, z;  // q
    double inv_m, k;    // 1/mq, 1/(mq (E_q + mq))
};
__device__ __forceinline__ BoostFrame boost_frame(const P4& q, double mq, double inv_m) {
    return {q.e, q.x, q.y, q.z, inv_m, 1.0 / (mq * (q.e + mq))};
}
__device__ __forceinline__ P4 boost_out(const P4& p, const BoostFrame& b) {
    double qp = b.x * p.x + b.y * p.y + b.z * p.z;
    double c = fma(qp, b.k, p.e * b.inv_m);
    return {(b.e * p.e + qp) * b.inv_m, p.x + b.x * c, p.y + b.y * c, p.z + b.z * c};
}
// The back-to-back daughters q1 = (e1, v) and q2 = (e2, -v) of a two-body decay, boosted out of
// the same frame: q2 . b = -(q1 . b) exactly, so the dot product is formed once.
__device__ __forceinline__ void boost_out_pair(const P4& q1, double e2, const BoostFrame& b, P4& p1, P4& p2) {
    const double qp = b.x * q1.x + b.y * q1.y + b.z * q1.z;
    const double c1 = fma(qp, b.k, q1.e * b.inv_m), c2 = fma(-qp, b.k, e2 * b.inv_m);
    p1 = {(b.e * q1.e + qp) * b.inv_m, q1.x + b.x * c1, q1.y + b.y * c1, q1.z + b.z * c1};
    p2 = {(b.e * e2 - qp) * b.inv_m, b.x * c2 - q1.x, b.y * c2 - q1.y, b.z * c2 - q1.z};
}
__device__ __forceinline__ P4 boost_in(const P4& p, const BoostFrame& b) {
    double qp = b.x * p.x + b.y * p.y + b.z * p.z;
    double c = fma(qp, b.k, -p.e * b.inv_m);
    return {(b.e * p.e - qp) * b.inv_m, p.x + b.x * c, p.y + b.y * c, p.z + b.z * c};
}

// Pure boost of p from the rest frame of q (invariant mass mq) to the frame where q is given.
__device__ __forceinline__ P4 boost_out(P4 p, P4 q, double mq) {
    double qp = q.x * p.x + q.y * p.y + q.z * p.z;
    double inv = 1.0 / mq;
    double c = qp / (mq * (q.e + mq)) + p.e * inv;
    return {(q.e * p.e + qp) * inv, p.x + q.x * c, p.y + q.y * c, p.z + q.z * c};
}

// The inverse boost: p given in the frame of q -> rest frame of q.
__device__ __forceinline__ P4 boost_in(P4 p, P4 q, double mq) {
    double qp = q.x * p.x + q.y * p.y + q.z * p.z;
    double inv = 1.0 / mq;
    double c = qp / (mq * (q.e + mq)) - p.e * inv;
    return {(q.e * p.e - qp) * inv, p.x + q.x * c, p.y + q.y * c, p.z + q.z * c};
}

// t range of a 2->2 block (Eq. t_invariant_theta): t = A + B cos(theta); the root of larger
// magnitude directly, the other from t+ t- =
//   (m1^2 - mA^2)(m2^2 - mB^2) + (m1^2 mB^2 - m2^2 mA^2)(m1^2 - m2^2 - mA^2 + mB^2)/s.
__device__ __forceinline__ void t_range(double s, double mA2, double mB2, double m1, double m2,
                                        double& tabs_min, double& tabs_max, double& B) {
    double m12 = m1 * m1, m22 = m2 * m2;
    double inv2s = 0.5 / s;
    double A = mA2 + m12 - (s + mA2 - mB2) * (s + m12 - m22) * inv2s;
    B = sqrt(kallen(s, mA2, mB2) * kallen_m(s, m1, m2)) * inv2s;
    double prod = (m12 - mA2) * (m22 - mB2) + (m12 * mB2 - m22 * mA2) * (m12 - m22 - mA2 + mB2) / s;
    const bool a_nonpos = nonpos_bits(A);       // A <= 0, on the bits
    double big = a_nonpos ? A - B : A + B;      // root without cancellation
    double small = !zero_bits(big) ? prod / big : 0.0;
    double tplus = a_nonpos ? small : big;      // closest to zero
    double tminus = a_nonpos ? big : small;
    tabs_min = -tplus;
    tabs_max = -tminus;
}

}  // namespace dev
}  // namespace ps
