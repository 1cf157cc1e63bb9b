// map_device.cuh -- device code of the phase-space interpreter: the invariant maps, decays and
// 2->2 blocks (FP64 and mixed forms), the slot-file frame and the op implementations.  Included
// by kernels.cu, and compiled at run time together with a channel's generated instruction list
// (jit.cpp), so it includes only headers that NVRTC can also read.
#pragma once

#include "kin.cuh"
#include "launch_params.h"
#include "philox.cuh"
#include "ps.h"
#include "tan_table.h"

namespace ps {
namespace dev {

using rng::philox4x32_10;
using rng::unit_from_bits;

// ---------------------------------------------------------------- azimuths
// cos and sin of 2 pi k / kTrigN into t[2k], t[2k+1], from sincospi (once per CTA)
__device__ __forceinline__ void stage_trig(double* t, int tid, int nthreads) {
    for (int k = tid; k < kTrigN; k += nthreads) {
        double s, c;
        sincospi(2.0 * k / kTrigN, &s, &c);
        t[2 * k] = c;
        t[2 * k + 1] = s;
    }
}

// sin and cos of phi = 2 pi r for r in [0, 1], table-driven: r kTrigN = k + f (exact; f in [0, 1)),
// x = f 2 pi / kTrigN < 0.0246, then sin x and cos x by their Taylor series to x^7 and x^6 (the
// first omitted terms are below 1e-17 of the result) and the angle-sum formulas with the
// tabulated point k.  About 15 FP64 operations where sincospi takes about 25; a few ulps.  Other r
// (outside [0, 1], NaN) take sincospi.
__device__ __forceinline__ void sincos_turn(double r, const double* trig, double& s, double& c) {
    if (static_cast<unsigned long long>(dbits(r)) > 0x3FF0000000000000ULL) {  // not in [+0, 1]
        sincospi(2.0 * r, &s, &c);
        return;
    }
    const double t = r * kTrigN;
    const int k = floor_small(t);
    const double f = t - small_to_double(k);
    const double x = f * (kPi / (kTrigN / 2)), x2 = x * x;
    const double sx = fma(x * x2, fma(x2, fma(x2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), x);
    const double cx = fma(x2, fma(x2, fma(x2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
    const int j = 2 * (k & (kTrigN - 1));  // r = 1 is the point k = 0 of the next turn
    const double ck = trig[j], sk = trig[j + 1];
    s = fma(sk, cx, ck * sx);
    c = fma(ck, cx, -(sk * sx));
}

// ---------------------------------------------------------------- tangent (Breit-Wigner map)
// tan x for |x| <= pi/4, table-driven: k = floor(|x| / h), h = pi/512, y = |x| - k h in [0, h)
// from a two-part (Cody-Waite) product, tan y by its Taylor series to y^7 (the next term is below
// 1e-19 of it), and the addition theorem as a correction of the tabulated point,
//   tan(k h + y) = tan(k h) + tan y (1 + tan^2 k h) / (1 - tan(k h) tan y),
// with tan(k h) a double-double and a non-negative correction (no cancellation).  Within 1.5 ulps,
// and the correctly rounded value for about 99 % of arguments (an emulation on the host against
// 80-bit tanl), in about 17 FP64 operations where tan takes about 29.  k is clamped to the table,
// so every argument reads inside it; beyond pi/4 the value is not the tangent (map_bw never
// passes one).
__device__ __forceinline__ double tan_quarter(double x) {
    const long long sign = dbits(x) & static_cast<long long>(0x8000000000000000ULL);
    const double ax = __longlong_as_double(dbits(x) ^ sign);
    const int k = min(floor_small(ax * kTanInvH), kTanN);
    const double kd = small_to_double(k);
    const double y = fma(-kd, kTanH2, fma(-kd, kTanH1, ax));
    const double y2 = y * y;
    const double p = fma(y2, fma(y2, 17.0 / 315.0, 2.0 / 15.0), 1.0 / 3.0);
    const double ty = fma(y * y2, p, y);
    const double th = __ldg(&kTanHi[k]);
    const double c = (ty * __ldg(&kTanSq1[k])) / fma(-th, ty, 1.0);
    const double t = th + (__ldg(&kTanLo[k]) + c);
    return __longlong_as_double(dbits(t) | sign);
}

// ---------------------------------------------------------------- invariant maps (Sec. 2.2.1)
// Power law G_nu / log map, anchored at x_min for nu <= 1 and at m^2 for nu > 1, so that
// 1 + z >= 1 and x - m^2 (and, for nu <= 1, x - x_min) keep full precision:
//   L = log1p((x_max - x_min)/lo), lo = x_min - m^2, hi = x_max - m^2, w = 1 - nu
//   nu == 1: x = x_min + lo expm1(r L),              J = (x - m^2) L
//   nu <  1: z = r expm1(w L),  x = x_min + lo expm1(log1p(z)/w),  J = (x - m^2) rho/(w (1+z))
//   nu >  1: z = (1-r) expm1(-w L), x - m^2 = hi exp(log1p(z)/w), J = -(x - m^2) rho'/(w (1+z))
__device__ __forceinline__ bool map_nu(double r, double m, double nu, double xmin, double xmax, double a,
                                       double& x, double& jac) {
    double m2 = pos_bits(m) ? m * m : -a;
    double lo = xmin - m2, hi = xmax - m2;
    bool ok = pos_bits(lo) && ge_pos_bits(hi, lo);
    double L = log1p((xmax - xmin) / lo);
    if (dbits(nu) == dbits(1.0)) {
        double e = expm1(r * L);
        double xm = fma(lo, e, lo);
        x = fma(lo, e, xmin);
        jac = xm * L;
    } else if (dbits(nu) < dbits(1.0)) {  // nu < 1 (nu is never NaN)
        double w = 1.0 - nu;
        double rho = expm1(w * L);
        double z = r * rho;
        double e = expm1(log1p(z) / w);
        double xm = fma(lo, e, lo);
        x = fma(lo, e, xmin);
        jac = xm * rho / (w * (1.0 + z));
    } else {
        double w = 1.0 - nu;
        double rho = expm1(-w * L);
        double z = (1.0 - r) * rho;
        double xm = hi * exp(log1p(z) / w);
        x = m2 + xm;
        jac = -xm * rho / (w * (1.0 + z));
    }
    x = clamp_nonneg(x, xmin, xmax);  // the map lands in [x_min, x_max] (rounding at the ends)
    if (!ok) { x = xmin; jac = 0.0; }
    return ok;
}

// Breit-Wigner G_BW with a = tan u1, b = tan u2, D = atan2(b - a, 1 + ab), u = u1 + D r.
// One tangent per event (tan_quarter) of the reduced angle arg (|arg| <= pi/4), chosen by
// selects, and each region's closed form written as num/den, so that one reciprocal serves every
// event of a warp and no region splits it:
//   u < -pi/4: arg = D r,     den = 1 - aT, x = x_min + mG T(1+a^2)/den, 1+tan^2u = (1+a^2)(1+T^2)/den^2
//   u >  pi/4: arg = D (1-r), den = 1 + bT, x = m^2 + mG (b-T)/den,      1+tan^2u = (1+b^2)(1+T^2)/den^2
//   otherwise: arg = u,       den = 1,      x = m^2 + mG T,              1+tan^2u = 1+T^2
// (tan u = (a + T)/(1 - aT), (b - T)/(1 + bT) and T; den > 0: a < -1 below, b > 1 above).
// J = D mG (1 + tan^2 u).  In the middle region 1/den = 1 exactly, so every region rounds as
// its own formula.  u1 = atan(a) may come in as the channel's constant (x_min immediate);
// have_u1 selects it.
__device__ __forceinline__ bool map_bw(double r, double M, double G, double xmin, double xmax,
                                       double& x, double& jac, bool have_u1 = false, double u1 = 0.0) {
    double mg = M * G, m2 = M * M;
    bool ok = pos_bits(mg) && ge_pos_bits(xmax, xmin);  // x_min >= 0 here (a squared mass)
    double inv_mg = 1.0 / mg;
    double a = (xmin - m2) * inv_mg, b = (xmax - m2) * inv_mg;
    double D = atan2((xmax - xmin) * inv_mg, fma(a, b, 1.0));
    double u = (have_u1 ? u1 : atan(a)) + D * r;
    bool low = below_neg_bits(u, 0.25 * kPi), high = above_pos_bits(u, 0.25 * kPi);
    double arg = low ? D * r : (high ? D * (1.0 - r) : u);
    double T = tan_quarter(arg);
    const double den = low ? 1.0 - a * T : (high ? 1.0 + b * T : 1.0);
    const double num = low ? T * (1.0 + a * a) : (high ? b - T : T);
    const double kk = low ? 1.0 + a * a : (high ? 1.0 + b * b : 1.0);
    const double rd = 1.0 / den;
    x = (low ? xmin : m2) + mg * (num * rd);
    jac = D * mg * (kk * (1.0 + T * T) * (rd * rd));
    x = clamp_nonneg(x, xmin, xmax);
    if (!ok) { x = xmin; jac = 0.0; }
    return ok;
}

// 2->2 block in (phi, t), Sec. 2.2.4: the polar axis is the direction of pA in the rest
// frame of p0 = pA + pB; cos(theta) from |t| via 1 -+ cos = (|t| - |t|_min)/B resp.
// (|t|_max - |t|)/B, whichever is smaller; the momentum is rotated by R(phi_A, theta_A)
// = Rz(phi_A) Ry(theta_A) (Sec. 2.2.6) and boosted back.
__device__ __forceinline__ double two_to_two(double rphi, P4 pA, P4 pB, double tabs, double m1, double m2,
                                             double s, double mA2, double mB2, P4& p1, P4& p2,
                                             const double* trig) {
    P4 p0 = p4_add(pA, pB);
    double m0 = sqrt(s);
    // 1/m0 = m0/s and the boost's 1/(m0 (E0 + m0)) from one division, R = 1/(s (E0 + m0))
    const double ep = p0.e + m0;
    const double R = 1.0 / (s * ep);
    const BoostFrame bf{p0.e, p0.x, p0.y, p0.z, m0 * (ep * R), m0 * R};
    P4 a = boost_in(pA, bf);
    double pt2 = a.x * a.x + a.y * a.y;
    bool has_pt = pos_bits(pt2);
    double ipt = has_pt ? rsqrt(pt2) : 0.0;
    double pt = pt2 * ipt;
    double rp = rsqrt(pt2 + a.z * a.z);
    double ca = a.z * rp, sa = pt * rp;
    double cpa = has_pt ? a.x * ipt : 1.0, spa = has_pt ? a.y * ipt : 0.0;

    double tlo, thi, B;
    t_range(s, mA2, mB2, m1, m2, tlo, thi, B);
    double dlo = tabs - tlo, dhi = thi - tabs;
    bool near_lo = dlo <= dhi;
    const bool b_pos = pos_bits(B);  // B > 0, on the bits
    double iB = b_pos ? 1.0 / B : 0.0;
    double first = (near_lo ? dlo : dhi) * iB;  // 1 - cos (near_lo) or 1 + cos
    double omc = b_pos ? (near_lo ? first : 2.0 - first) : 1.0;
    double opc = b_pos ? (near_lo ? 2.0 - first : first) : 1.0;
    double cth = (omc <= opc) ? 1.0 - omc : opc - 1.0;
    const double so = omc * opc;
    double sth = sqrt(pos_bits(so) ? so : 0.0);
    double sph, cph;
    sincos_turn(rphi, trig, sph, cph);

    double m12 = m1 * m1, m22 = m2 * m2;
    double i2m0 = 0.5 * bf.inv_m;
    double pabs = sqrt(kallen_m(s, m1, m2)) * i2m0;
    double e1 = (s + m12 - m22) * i2m0, e2 = (s + m22 - m12) * i2m0;
    double vx = pabs * sth * cph, vy = pabs * sth * sph, vz = pabs * cth;
    // Ry(theta_A) then Rz(phi_A)
    double rx = ca * vx + sa * vz, rz = -sa * vx + ca * vz;
    P4 q1 = {e1, cpa * rx - spa * vy, spa * rx + cpa * vy, rz};
    boost_out_pair(q1, e2, bf, p1, p2);
    return 0.5 * kPi * rsqrt(kallen(s, mA2, mB2));
}

// 1->2 decay in (phi, theta), Sec. 2.2.3: cos = 2 r_theta - 1, sin = 2 sqrt(r_theta (1 - r_theta)),
// phi = 2 pi r_phi, built at rest and optionally boosted to the frame of p0.
template <bool kBoost>
__device__ __forceinline__ double two_body(double rphi, double rth, double s0, double m1, double m2, P4 p0,
                                           P4& p1, P4& p2, const double* trig) {
    double m0 = sqrt(s0);
    // 1/s0 by its own division: the Jacobian sqrt(lambda)/s0 must not pick up the rounding of the
    // parent's energy (as a reciprocal shared with the boost's 1/(m0 (E0 + m0)) would)
    const double inv_s0 = 1.0 / s0;
    const double inv_m0 = m0 * inv_s0;  // 1/m0 = m0/s0
    double m12 = m1 * m1, m22 = m2 * m2;
    // sqrt(lambda) = s0 exactly for two massless daughters
    double sl = (zero_bits(m12) && zero_bits(m22)) ? s0 : sqrt(kallen_m(s0, m1, m2));
    double i2m0 = 0.5 * inv_m0;
    double pabs = sl * i2m0;
    double e1 = (s0 + m12 - m22) * i2m0, e2 = (s0 + m22 - m12) * i2m0;
    double cth = 2.0 * rth - 1.0;
    double sth = 2.0 * sqrt(rth * (1.0 - rth));
    double sph, cph;
    sincos_turn(rphi, trig, sph, cph);
    P4 q1 = {e1, pabs * sth * cph, pabs * sth * sph, pabs * cth};
    P4 q2 = {e2, -q1.x, -q1.y, -q1.z};
    if (kBoost) {
        boost_out_pair(q1, e2, boost_frame(p0, m0, inv_m0), p1, p2);
    } else {
        p1 = q1;
        p2 = q2;
    }
    return 0.5 * kPi * sl * inv_s0;
}

// ---------------------------------------------------------------- interpreter
struct Frame {
    static constexpr bool kStatic = false;  // slots addressed at run time
    double* S;            // slot file base for this thread: slot k at S[k * block]
    const double* imm;    // channel immediates (shared memory)
    int block;
    const float* immf;    // the immediates rounded to float (mixed kernel only)
};

__device__ __forceinline__ double ld(const Frame& f, int a) { return a >= 0 ? f.S[a * f.block] : f.imm[~a]; }
__device__ __forceinline__ void st(const Frame& f, int slot, double v) { f.S[slot * f.block] = v; }
__device__ __forceinline__ P4 ldp(const Frame& f, int a) {
    const double* q = f.S + a * f.block;
    return {q[0], q[f.block], q[2 * f.block], q[3 * f.block]};
}
__device__ __forceinline__ void stp(const Frame& f, int slot, P4 p) {
    double* q = f.S + slot * f.block;
    q[0] = p.e;
    q[f.block] = p.x;
    q[2 * f.block] = p.y;
    q[3 * f.block] = p.z;
}

// Loops of an op over its arguments.  For a register frame, whose slots must be indexed by
// constants, the loop is fully unrolled: its bounds are constants once the generated instruction
// list is inlined.  The shared-memory frame keeps a plain loop.
template <class Fr, class F>
__device__ __forceinline__ void op_loop(int b, int e, int step, F&& body) {
    if constexpr (Fr::kStatic) {
#pragma unroll
        for (int j = b; j < e; j += step) body(j);
    } else {
        for (int j = b; j < e; j += step) body(j);
    }
}
// body(i) for every set bit i < nbits of mask
template <class Fr, class F>
__device__ __forceinline__ void op_bits(int mask, int nbits, F&& body) {
    if constexpr (Fr::kStatic) {
#pragma unroll
        for (int i = 0; i < nbits; ++i)
            if ((mask >> i) & 1) body(i);
    } else {
        while (mask) {
            const int i = __ffs(mask) - 1;
            mask &= mask - 1;
            body(i);
        }
    }
}

// ---------------------------------------------------------------- register frame
// A compiled channel (jit.cpp) keeps its slot file in registers: RegFrame<NS, Imm> holds NS slots
// and reads immediates from the compile-time functions Imm::v(i), Imm::f(i).  Every access is
// by a constant index once the generated instruction list is inlined, so the array lives in
// registers.  Mixed-precision momenta are held as the doubles of their float components.
template <int NS, class Imm>
struct RegFrame {
    static constexpr bool kStatic = true;
    mutable double v[NS > 0 ? NS : 1];
};
template <int NS, class Imm>
__device__ __forceinline__ double ld(const RegFrame<NS, Imm>& f, int a) { return a >= 0 ? f.v[a] : Imm::v(~a); }
template <int NS, class Imm>
__device__ __forceinline__ void st(const RegFrame<NS, Imm>& f, int slot, double x) { f.v[slot] = x; }
template <int NS, class Imm>
__device__ __forceinline__ P4 ldp(const RegFrame<NS, Imm>& f, int a) { return {f.v[a], f.v[a + 1], f.v[a + 2], f.v[a + 3]}; }
template <int NS, class Imm>
__device__ __forceinline__ void stp(const RegFrame<NS, Imm>& f, int slot, P4 p) {
    f.v[slot] = p.e;
    f.v[slot + 1] = p.x;
    f.v[slot + 2] = p.y;
    f.v[slot + 3] = p.z;
}
// Small integers held as immediates (counts, kinds, masks): decoded from their bits for the
// shared-memory frame (integer ALU), by a conversion for a register frame, where they are
// compile-time constants that the conversion folds away (the bit decode would stay opaque).
template <class Fr>
__device__ __forceinline__ int op_int(double v) {
    if constexpr (Fr::kStatic) return static_cast<int>(v);
    else return small_int(v);
}

// One propagator denominator of an SDE channel weight (Sec. 2.1): kind 1 a t-channel 1/(t - M^2)^2,
// kind 0 an s-channel 1/((s - M^2)^2 + M^2 Gamma^2); the product is kept in range by dividing
// it out into P.  P_j = P / den at the end.
// The factor from the invariant s = q^2 (a compiled channel computes each distinct invariant once
// and shares it between the channels whose propagators use it).
__device__ __forceinline__ void sde_factor_s(double& den, double& P, double s, int kind, double M, double G) {
    const double d = s - M * M, mg = M * G;
    den *= (kind == 1) ? d * d : fma(d, d, mg * mg);
    if (above_pos_bits(den, 1e200)) {  // keep the running product in range
        P /= den;
        den = 1.0;
    }
}
__device__ __forceinline__ void sde_factor(double& den, double& P, const P4& q, int kind, double M, double G) {
    sde_factor_s(den, P, p4_sq(q), kind, M, G);
}

// A channel's VEGAS grid in shared memory: dims rows of bins + 1 edges, then dims rows of bins
// widths e[k+1] - e[k], each the difference the lookup would form (in the staged precision, T
// double or float), computed once per CTA and channel instead of once per event and dimension.
template <class T>
__device__ __forceinline__ void stage_grid(T* s, const double* g, int dims, int bins, int tid, int nthreads) {
    const int ng = dims * (bins + 1);
    for (int i = tid; i < ng; i += nthreads) s[i] = static_cast<T>(g[i]);
    for (int i = tid; i < dims * bins; i += nthreads) {
        const int j = i / bins, k = i % bins;
        s[ng + i] = static_cast<T>(g[j * (bins + 1) + k + 1]) - static_cast<T>(g[j * (bins + 1) + k]);
    }
}

// One instruction of the FP64 interpreter on frame Fr (the shared-memory slot file of the
// interpreter kernel, or the register frame of a compiled channel).  grid: the channel's staged
// VEGAS grid in shared memory, preceded by the azimuth table (grid - kTrigDoubles).
template <class Fr>
__device__ __forceinline__ void exec_op(const int op, const int32_t* a, const int32_t* o, const int na, const int no,
                                        const Fr& f, const double* grid, int vbins, unsigned long long* cut_count,
                                        bool active) {
        switch (op) {
            case PS_OP_VEGAS: {
                double jac = 1.0;
                const double nb = small_to_double(vbins);
                // with a power-of-two bin count, prod_j (nb w_j) = (prod_j w_j) nb^na exactly (scaling
                // by a power of two commutes with rounding): one multiply by nb^na, from its bits
                const int q = __ffs(vbins) - 1;
                const bool pow2 = (vbins & (vbins - 1)) == 0 && q * na <= 1000;
                op_loop<Fr>(0, na, 1, [&](int j) {
                    double r = ld(f, a[j]);
                    double rn = r * nb;
                    // the bin and its double from the bits (no FP64-pipe conversions)
                    int k = min(floor_small(rn), vbins - 1);
                    k = max(k, 0);
                    const double e0 = grid[j * (vbins + 1) + k];
                    const double wdt = grid[na * (vbins + 1) + j * vbins + k];  // staged e[k+1] - e[k]
                    st(f, o[j], fma(rn - small_to_double(k), wdt, e0));
                    jac *= pow2 ? wdt : nb * wdt;
                });
                if (pow2) jac *= __longlong_as_double(static_cast<long long>(1023 + q * na) << 52);
                st(f, o[na], jac);
                break;
            }
            case PS_OP_INVARIANT_NU: {
                double x, j;
                map_nu(ld(f, a[0]), ld(f, a[1]), ld(f, a[2]), ld(f, a[3]), ld(f, a[4]), ld(f, a[5]), x, j);
                st(f, o[0], x);
                st(f, o[1], j);
                break;
            }
            case PS_OP_INVARIANT_BW: {
                double x, j;
                map_bw(ld(f, a[0]), ld(f, a[1]), ld(f, a[2]), ld(f, a[3]), ld(f, a[4]), x, j, na > 5,
                       na > 5 ? ld(f, a[5]) : 0.0);
                st(f, o[0], x);
                st(f, o[1], j);
                break;
            }
            case PS_OP_R_TO_X1X2: {
                double r = ld(f, a[0]), shat = ld(f, a[1]), S = ld(f, a[2]);
                // 1/S once (a constant that a compiled program folds; S is the collider's), then
                // products in place of the two divisions by S
                const double iS = 1.0 / S;
                const double tau = shat * iS;
                double L = log(tau);
                const double l1 = r * L, l2 = (1.0 - r) * L;  // log x1, log x2
                const double x1 = exp(l1);
                st(f, o[0], x1);
                st(f, o[1], tau / x1);  // x1 x2 = tau: a division where a second exponential was
                st(f, o[2], -L * iS);
                if (no > 3) {
                    st(f, o[3], l1);
                    st(f, o[4], l2);
                }
                break;
            }
            case PS_OP_COM_P_IN: {
                double h = 0.5 * ld(f, a[0]);
                stp(f, o[0], P4{h, 0.0, 0.0, h});
                stp(f, o[1], P4{h, 0.0, 0.0, -h});
                break;
            }
            case PS_OP_T_INV_MIN_MAX: {
                double lo, hi, B;
                t_range(ld(f, a[0]), ld(f, a[1]), ld(f, a[2]), ld(f, a[3]), ld(f, a[4]), lo, hi, B);
                st(f, o[0], lo);
                st(f, o[1], hi);
                break;
            }
            case PS_OP_TWO_TO_TWO_COM: {
                P4 p1, p2;
                double j = two_to_two(ld(f, a[0]), ldp(f, a[1]), ldp(f, a[2]), ld(f, a[3]), ld(f, a[4]),
                                      ld(f, a[5]), ld(f, a[6]), ld(f, a[7]), ld(f, a[8]), p1, p2,
                                      grid - kTrigDoubles);
                stp(f, o[0], p1);
                stp(f, o[1], p2);
                st(f, o[2], j);
                break;
            }
            case PS_OP_TWO_BODY_DECAY: {
                P4 p1, p2;
                double j = two_body<true>(ld(f, a[0]), ld(f, a[1]), ld(f, a[2]), ld(f, a[3]), ld(f, a[4]),
                                          ldp(f, a[5]), p1, p2, grid - kTrigDoubles);
                stp(f, o[0], p1);
                stp(f, o[1], p2);
                st(f, o[2], j);
                break;
            }
            case PS_OP_TWO_BODY_DECAY_COM: {
                P4 p1, p2;
                double j = two_body<false>(ld(f, a[0]), ld(f, a[1]), ld(f, a[2]), ld(f, a[3]), ld(f, a[4]),
                                           P4{0, 0, 0, 0}, p1, p2, grid - kTrigDoubles);
                stp(f, o[0], p1);
                stp(f, o[1], p2);
                st(f, o[2], j);
                break;
            }
            case PS_OP_BOOST_BEAM: {
                // light-cone form of the longitudinal boost: E+p_z scales by rho = sqrt(x1/x2),
                // E-p_z by 1/rho (no cancellation for extreme boosts)
                double x1 = ld(f, a[na - 2]), x2 = ld(f, a[na - 1]);
                const double t = rsqrt(x1 * x2);  // rho = sqrt(x1/x2) = x1 t, 1/rho = x2 t
                double rho = x1 * t;
                double irho = x2 * t;
                op_loop<Fr>(0, na - 2, 1, [&](int k) {
                    P4 p = ldp(f, a[k]);
                    double plus = rho * (p.e + p.z), minus = (p.e - p.z) * irho;
                    stp(f, o[k], P4{0.5 * (plus + minus), p.x, p.y, 0.5 * (plus - minus)});
                });
                break;
            }
            case PS_OP_REDUCE_PRODUCT: {
                double v = ld(f, a[0]);
                op_loop<Fr>(1, na, 1, [&](int k) { v *= ld(f, a[k]); });
                st(f, o[0], v);
                break;
            }
            case PS_OP_CUT_UNPHYSICAL: {
                double w = ld(f, a[0]), x1 = ld(f, a[1]), x2 = ld(f, a[2]);
                bool bad = !finite_bits(w) || !(in_unit_bits(x1) && in_unit_bits(x2));
                op_loop<Fr>(3, na, 1, [&](int k) {
                    P4 p = ldp(f, a[k]);
                    bad |= !(finite_bits(p.e) && finite_bits(p.x) && finite_bits(p.y) && finite_bits(p.z));
                });
                if (bad && active) atomicAdd(cut_count, 1ULL);
                st(f, o[0], bad ? 0.0 : w);
                break;
            }
            case PS_OP_ADD: st(f, o[0], ld(f, a[0]) + ld(f, a[1])); break;
            case PS_OP_SUB: st(f, o[0], ld(f, a[0]) - ld(f, a[1])); break;
            case PS_OP_MUL: st(f, o[0], ld(f, a[0]) * ld(f, a[1])); break;
            case PS_OP_DIV: st(f, o[0], ld(f, a[0]) / ld(f, a[1])); break;
            case PS_OP_SQRT: st(f, o[0], sqrt(ld(f, a[0]))); break;
            case PS_OP_SQUARE: { double v = ld(f, a[0]); st(f, o[0], v * v); break; }
            case PS_OP_MAX: st(f, o[0], fmax_bits(ld(f, a[0]), ld(f, a[1]))); break;
            case PS_OP_MOM_ADD: stp(f, o[0], p4_add(ldp(f, a[0]), ldp(f, a[1]))); break;
            case PS_OP_MOM_SUB: stp(f, o[0], p4_sub(ldp(f, a[0]), ldp(f, a[1]))); break;
            case PS_OP_PDF_POWER: {
                // one density, or the pair f(x1) f(x2) = exp(alpha (log x1 + log x2)) (1-x1)^b (1-x2)^b
                const bool pair = na == 6;
                double x = ld(f, a[0]), al = ld(f, a[1]), be = ld(f, a[2]);
                double lx = na > 3 ? ld(f, a[3]) : log(x);
                // an add that is never contracted with the product forming log x2 (a compiled
                // program could fuse them; the interpreter's slot file rounds the product)
                if (pair) lx = __dadd_rn(lx, ld(f, a[5]));
                double fx = exp(al * lx);
                auto pw = [&](double y) {
                    if (be == 3.0) return y * y * y;
                    if (be == 2.0) return y * y;
                    if (be == 1.0) return y;
                    if (be == 0.0) return 1.0;
                    return pow(y, be);
                };
                double fy = pw(1.0 - x);
                if (pair) fy *= pw(1.0 - ld(f, a[4]));
                st(f, o[0], fx * fy);
                break;
            }
            case PS_OP_PROPAGATOR: {
                double s = ld(f, a[0]), M = ld(f, a[1]), G = ld(f, a[2]);
                double d = s - M * M;
                st(f, o[0], 1.0 / (d * d + M * M * G * G));
                break;
            }
            case PS_OP_ONE_PLUS_COS2: {
                P4 p = ldp(f, a[0]);
                double c2 = p.z * p.z / (p.x * p.x + p.y * p.y + p.z * p.z);
                st(f, o[0], 1.0 + c2);
                break;
            }
            case PS_OP_CHANNEL_WEIGHT: {
                // P_j = 1 / prod(denominators): one division per channel; kind and mask decoded
                // from their bits, the momentum sum over the set bits of the mask only
                const int k = op_int<Fr>(ld(f, a[0]));
                const P4 pa = ldp(f, a[1]);
                double den = 1.0, P = 1.0;
                op_loop<Fr>(2 + k, na - 3, 4, [&](int j) {
                    const int kind = op_int<Fr>(ld(f, a[j]));
                    const int mask = op_int<Fr>(ld(f, a[j + 1]));
                    const double M = ld(f, a[j + 2]), G = ld(f, a[j + 3]);
                    P4 q = (kind == 1) ? pa : P4{0.0, 0.0, 0.0, 0.0};
                    op_bits<Fr>(mask, k, [&](int i) {
                        q = (kind == 1) ? p4_sub(q, ldp(f, a[2 + i])) : p4_add(q, ldp(f, a[2 + i]));
                    });
                    sde_factor(den, P, q, kind, M, G);
                });
                st(f, o[0], P / den);
                break;
            }
            default: break;
        }
}

// Executes one channel's instruction list for the calling thread's event.
static __device__ void run_code(const int32_t* code, int len, const Frame& f, const double* grid, int vbins,
                         unsigned long long* cut_count, bool active) {
    int pc = 0;
    while (pc < len) {
        const int op = code[pc], na = code[pc + 1], no = code[pc + 2];
        const int32_t* a = code + pc + 3;
        exec_op(op, a, a + na, na, no, f, grid, vbins, cut_count, active);
        pc += 3 + na + no;
    }
}


// ================================================================ mixed precision
// PS_PRECISION_MIXED: bulk kinematics in FP32 (momenta are carried as float in the slot file,
// angles, boosts, rotations, transcendentals of the maps, parton densities), FP64 kept for the
// islands that are sensitive to cancellation: invariant assembly x = x_min + lo e and s - m^2,
// the Kallen function at threshold, the t range and 1 - cos(theta) for small |t|, the s-order
// bounds, and every Jacobian product.  Scalars stay FP64 in the slot file.
namespace mx {

// Conversions between binary64 and binary32 written on the IEEE 754 bit layouts and executed by
// the integer ALU.  The FP64 pipe that bounds these kernels also executes the hardware
// conversions, and the mixed form converts at every edge of an FP64 island; on the integer
// ALU a conversion costs issue slots of a pipe with 32 times the FP64 pipe's rate.  Both give
// the correctly rounded result (round to nearest, ties to even) for every input; NaN comes out
// as a NaN.
__device__ __forceinline__ double f2d(float x) {
    const uint32_t u = __float_as_uint(x), a = u & 0x7FFFFFFFu;
    uint32_t hi, lo = u << 29;  // the low three fraction bits open the low word
    if (__builtin_expect(a - 0x00800000u < 0x7F000000u, 1)) {
        hi = (a >> 3) + 0x38000000u;  // normal: exponent rebiased 127 -> 1023 (+896 << 20)
    } else if (a >= 0x7F800000u) {
        hi = 0x7FF00000u | ((a >> 3) & 0xFFFFFu);  // infinity, NaN
    } else if (a != 0u) {
        const int lz = __clz(a);                    // subnormal: leading bit at 31 - lz (9..31)
        const uint32_t m = a << (lz - 8);           // ... moved to bit 23
        hi = (static_cast<uint32_t>(905 - lz) << 20) | ((m >> 3) & 0xFFFFFu);  // 2^(8 - lz - 126)
        lo = m << 29;
    } else {
        hi = 0u;
    }
    return __hiloint2double(static_cast<int>((u & 0x80000000u) | hi), static_cast<int>(lo));
}

__device__ __forceinline__ float d2f(double x) {
    const uint32_t hi = static_cast<uint32_t>(__double2hiint(x)), lo = static_cast<uint32_t>(__double2loint(x));
    const uint32_t e = (hi >> 20) & 0x7FFu;
    uint32_t r;
    if (__builtin_expect(e - 897u < 254u, 1)) {  // a float normal: 23 fraction bits, rounded
        const uint32_t m = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu, rem = lo & 0x1FFFFFFFu;
        const uint32_t up = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
        r = ((e - 896u) << 23) + m + up;  // a carry out of the fraction raises the exponent
    } else if (e >= 1151u) {              // beyond the float range, infinity, NaN
        r = (e == 0x7FFu && ((hi & 0xFFFFFu) | lo) != 0u) ? 0x7FFFFFFFu : 0x7F800000u;
    } else if (e >= 873u) {               // a float subnormal: the 53-bit significand shifted
        const unsigned long long sig =
            (1ULL << 52) | (static_cast<unsigned long long>(hi & 0xFFFFFu) << 32) | lo;
        const int sh = static_cast<int>(926u - e);  // to units of 2^-149: 30..53
        const unsigned long long q = sig >> sh, rem = sig & ((1ULL << sh) - 1ULL), half = 1ULL << (sh - 1);
        r = static_cast<uint32_t>(q) + ((rem > half || (rem == half && (q & 1ULL))) ? 1u : 0u);
    } else {
        r = 0u;  // zero, or below half the least subnormal
    }
    return __uint_as_float((hi & 0x80000000u) | r);
}

// FP32 seeds from IEEE operations only (a compile-time evaluation of a constant argument gives
// the device's bits, so compiled and interpreted programs agree):
// 1/sqrt(m), m in [1, 4): the bit-level estimate 0x5F375A86 - (bits >> 1) (Lomont 2003,
// relative error below 3.5%) and three Newton steps y (3/2 - m y^2 / 2);
// 1/m, m in [1, 2): the linear estimate 24/17 - 8/17 m (the minimax line of the Newton-Raphson
// division, error below 1/17) and three Newton steps y + y (1 - m y).  Both end within a few
// float ulps.
__device__ __forceinline__ float rsqrt_m(float m) {
    float y = __uint_as_float(0x5F375A86u - (__float_as_uint(m) >> 1));
    const float h = 0.5f * m;
    y = y * fmaf(-h, y * y, 1.5f);
    y = y * fmaf(-h, y * y, 1.5f);
    return y * fmaf(-h, y * y, 1.5f);
}
__device__ __forceinline__ float rcp_m(float m) {
    float y = fmaf(-8.0f / 17.0f, m, 24.0f / 17.0f);
    y = fmaf(y, fmaf(-m, y, 1.0f), y);
    y = fmaf(y, fmaf(-m, y, 1.0f), y);
    return fmaf(y, fmaf(-m, y, 1.0f), y);
}

struct F4 {
    float e, x, y, z;
};

__device__ __forceinline__ F4 f4_add(F4 a, F4 b) { return {a.e + b.e, a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ F4 f4_sub(F4 a, F4 b) { return {a.e - b.e, a.x - b.x, a.y - b.y, a.z - b.z}; }

// float momentum in 4 consecutive slots (low half of each 8-byte slot)
__device__ __forceinline__ F4 ldp(const Frame& f, int a) {
    const float* q = reinterpret_cast<const float*>(f.S + a * f.block);
    const int st = 2 * f.block;
    return {q[0], q[st], q[2 * st], q[3 * st]};
}
__device__ __forceinline__ void stp(const Frame& f, int slot, F4 p) {
    float* q = reinterpret_cast<float*>(f.S + slot * f.block);
    const int st = 2 * f.block;
    q[0] = p.e;
    q[st] = p.x;
    q[2 * st] = p.y;
    q[3 * st] = p.z;
}
// immediates come from their float copy: no conversion per read
__device__ __forceinline__ float ldf(const Frame& f, int a) { return a >= 0 ? d2f(f.S[a * f.block]) : f.immf[~a]; }
// a float result into a scalar slot (held as its double in the shared-memory slot file)
__device__ __forceinline__ void stf(const Frame& f, int slot, float x) { f.S[slot * f.block] = f2d(x); }

// Seeds of the FP64 reciprocal square root and reciprocal for any normal double x = 1.f 2^e:
// the exponent is split off on the integer ALU, the FP32 seed sees only the fraction
// (truncated to 23 bits) with an exponent of 0 or 1, and the result's exponent is set from e.
// Relative error below ~2.5e-7 (the truncation and the FP32 rounding).
__device__ __forceinline__ double rsqrt_seed(double x) {  // x > 0
    const uint32_t hi = static_cast<uint32_t>(__double2hiint(x)), lo = static_cast<uint32_t>(__double2loint(x));
    const int e = static_cast<int>((hi >> 20) & 0x7FFu) - 1023;
    const int p = e & 1, k = (e - p) / 2;  // x = 1.f 2^p 4^k: rsqrt(x) = rsqrt(1.f 2^p) 2^-k
    const float r =
        rsqrt_m(__uint_as_float((static_cast<uint32_t>(127 + p) << 23) | (__funnelshift_l(lo, hi, 3) & 0x7FFFFFu)));
    const uint32_t u = __float_as_uint(r);  // in (1/2, 1]
    return __hiloint2double(static_cast<int>((u >> 3) + 0x38000000u - (static_cast<uint32_t>(k) << 20)),
                            static_cast<int>(u << 29));
}
__device__ __forceinline__ double rcp_seed(double x) {  // x != 0
    const uint32_t hi = static_cast<uint32_t>(__double2hiint(x)), lo = static_cast<uint32_t>(__double2loint(x));
    const int e = static_cast<int>((hi >> 20) & 0x7FFu) - 1023;
    const float r = rcp_m(__uint_as_float(0x3F800000u | (__funnelshift_l(lo, hi, 3) & 0x7FFFFFu)));
    const uint32_t u = __float_as_uint(r);  // 1/(1.f) in (1/2, 1]
    return __hiloint2double(
        static_cast<int>((hi & 0x80000000u) | ((u >> 3) + 0x38000000u - (static_cast<uint32_t>(e) << 20))),
        static_cast<int>(u << 29));
}

// sqrt in FP64 from the reciprocal-square-root seed and one Newton step in FP64:
// s = x r, e = x - s^2, s += e r/2 (relative error ~ 1.5 delta^2 for a seed error delta:
// below 1e-13).  0 for x <= 0 and NaN; x a normal double otherwise.  The empty asm makes x
// opaque: a compiled program evaluates sqrt64 of a constant at run time, as the interpreter
// does, so that no folded result changes how the expressions around it are contracted.
__device__ __forceinline__ double sqrt64(double x) {
    asm("" : "+d"(x));
    if (!pos_bits(x)) return 0.0;
    double r = rsqrt_seed(x);
    double s = x * r;
    double e = fma(-s, s, x);
    return fma(e, 0.5 * r, s);
}

// 1/x in FP64 from the reciprocal seed and one Newton step (relative error ~ delta^2), for a
// normal double x.
__device__ __forceinline__ double rcp64(double x) {
    asm("" : "+d"(x));  // opaque, as in sqrt64
    double r = rcp_seed(x);
    double e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// lambda(x, m1^2, m2^2) from the masses m1, m2 >= 0 (the factorised form, no square roots)
__device__ __forceinline__ double kallen64_m(double x, double m1, double m2) {
    double l;
    if (zero_bits(m1 * m1) && zero_bits(m2 * m2)) {
        l = x * x;
    } else {
        double hi = m1 + m2, lo = m1 - m2;
        l = fma(-hi, hi, x) * fma(-lo, lo, x);  // explicit: the same roundings with constant masses
    }
    return pos_bits(l) ? l : 0.0;
}

__device__ __forceinline__ double kallen64(double x, double y, double z) {
    double l;
    if (zero_bits(y) && zero_bits(z)) {
        l = x * x;
    } else if (nonneg_bits(y) && nonneg_bits(z)) {
        // explicit FMAs: with constant masses a compiled program folds sqrt64(y) and sqrt64(z),
        // and the contraction of x - hi^2 must not depend on it
        double ry = sqrt64(y), rz = sqrt64(z);
        double hi = ry + rz, lo = ry - rz;
        l = fma(-hi, hi, x) * fma(-lo, lo, x);
    } else if (nonpos_bits(y) && nonpos_bits(z)) {
        double d = z - y;
        l = x * x - 2.0 * x * (y + z) + d * d;
    } else {
        double d = x - y - z;
        l = d * d - 4.0 * y * z;
    }
    return pos_bits(l) ? l : 0.0;
}

__device__ __forceinline__ F4 boost_out(F4 p, F4 q, float mq) {
    float qp = q.x * p.x + q.y * p.y + q.z * p.z;
    float inv = 1.0f / mq;
    float c = qp / (mq * (q.e + mq)) + p.e * inv;
    return {(q.e * p.e + qp) * inv, p.x + q.x * c, p.y + q.y * c, p.z + q.z * c};
}
__device__ __forceinline__ F4 boost_in(F4 p, F4 q, float mq) {
    float qp = q.x * p.x + q.y * p.y + q.z * p.z;
    float inv = 1.0f / mq;
    float c = qp / (mq * (q.e + mq)) - p.e * inv;
    return {(q.e * p.e - qp) * inv, p.x + q.x * c, p.y + q.y * c, p.z + q.z * c};
}

// power law / log map: transcendentals in float, x = x_min + lo e assembled in FP64
__device__ __forceinline__ void map_nu(float r, double m, double nu, double xmin, double xmax, double a,
                                       double& x, double& jac) {
    double m2 = pos_bits(m) ? m * m : -a;
    double lo = xmin - m2, hi = xmax - m2;
    bool ok = pos_bits(lo) && ge_pos_bits(hi, lo);
    float L = log1pf(d2f(xmax - xmin) / d2f(lo));
    float e, jf;
    if (dbits(nu) == dbits(1.0)) {
        e = expm1f(r * L);
        jf = (1.0f + e) * L;
        x = fma(lo, f2d(e), xmin);
        jac = lo * f2d(jf);
    } else if (dbits(nu) < dbits(1.0)) {  // nu < 1 (nu is never NaN)
        float w = d2f(1.0 - nu);
        float rho = expm1f(w * L);
        float z = r * rho;
        e = expm1f(log1pf(z) / w);
        jf = (1.0f + e) * rho / (w * (1.0f + z));
        x = fma(lo, f2d(e), xmin);
        jac = lo * f2d(jf);
    } else {
        float w = d2f(1.0 - nu);
        float rho = expm1f(-w * L);
        float z = (1.0f - r) * rho;
        float g = expf(log1pf(z) / w);
        double xm = hi * f2d(g);
        x = m2 + xm;
        jac = -xm * f2d(rho / (w * (1.0f + z)));
    }
    x = clamp_nonneg(x, xmin, xmax);
    if (!ok) { x = xmin; jac = 0.0; }
}

// Breit-Wigner: angles and tan in float (the same endpoint-relative regions as the FP64 form, as
// one num/den chosen by selects with a single reciprocal), s - m^2 and the assembly of x in FP64
__device__ __forceinline__ void map_bw(float r, double M, double G, double xmin, double xmax, double& x, double& jac,
                                       bool have_u1 = false, double u1 = 0.0) {
    double mg = M * G, m2 = M * M;
    bool ok = pos_bits(mg) && ge_pos_bits(xmax, xmin);  // x_min >= 0 here (a squared mass)
    float mgf = d2f(mg);
    float imgf = 1.0f / mgf;
    float a = d2f(xmin - m2) * imgf, b = d2f(xmax - m2) * imgf;
    float D = atan2f(d2f(xmax - xmin) * imgf, fmaf(a, b, 1.0f));
    float u = (have_u1 ? d2f(u1) : atanf(a)) + D * r;
    bool low = u < -0.785398163f, high = u > 0.785398163f;
    float arg = low ? D * r : (high ? D * (1.0f - r) : u);
    float T = tanf(arg);
    const float den = low ? 1.0f - a * T : (high ? 1.0f + b * T : 1.0f);
    const float num = low ? T * (1.0f + a * a) : (high ? b - T : T);
    const float kk = low ? 1.0f + a * a : (high ? 1.0f + b * b : 1.0f);
    const float rd = 1.0f / den;  // 1 exactly in the middle region
    x = (low ? xmin : m2) + f2d(mgf * (num * rd));
    const float sec2 = kk * (1.0f + T * T) * (rd * rd);
    jac = f2d(D * mgf * sec2);
    x = clamp_nonneg(x, xmin, xmax);
    if (!ok) { x = xmin; jac = 0.0; }
}

// t range: FP64 island (small |t|), with the fast sqrt/reciprocal
__device__ __forceinline__ void t_range(double s, double mA2, double mB2, double m1, double m2, double& tabs_min,
                                        double& tabs_max, double& B) {
    double m12 = m1 * m1, m22 = m2 * m2;
    double is = rcp64(s);
    double A = mA2 + m12 - 0.5 * (s + mA2 - mB2) * (s + m12 - m22) * is;
    B = 0.5 * sqrt64(kallen64(s, mA2, mB2) * kallen64_m(s, m1, m2)) * is;
    double prod = (m12 - mA2) * (m22 - mB2) + (m12 * mB2 - m22 * mA2) * (m12 - m22 - mA2 + mB2) * is;
    const bool a_nonpos = nonpos_bits(A);  // A <= 0, on the bits
    double big = a_nonpos ? A - B : A + B;
    double small = !zero_bits(big) ? prod * rcp64(big) : 0.0;
    tabs_min = -(a_nonpos ? small : big);
    tabs_max = -(a_nonpos ? big : small);
}

__device__ __forceinline__ double two_to_two(float rphi, F4 pA, F4 pB, double tabs, double m1, double m2, double s,
                                             double mA2, double mB2, F4& p1, F4& p2) {
    F4 p0 = f4_add(pA, pB);
    float m0 = d2f(sqrt64(s));
    F4 a = boost_in(pA, p0, m0);
    float pt = sqrtf(a.x * a.x + a.y * a.y);
    float rp = rsqrtf(pt * pt + a.z * a.z);
    float ca = a.z * rp, sa = pt * rp;
    bool has_pt = pt > 0.0f;
    float ipt = has_pt ? 1.0f / pt : 0.0f;
    float cpa = has_pt ? a.x * ipt : 1.0f, spa = has_pt ? a.y * ipt : 0.0f;
    double tlo, thi, B;
    t_range(s, mA2, mB2, m1, m2, tlo, thi, B);
    double dlo = tabs - tlo, dhi = thi - tabs;
    bool near_lo = dlo <= dhi;
    const bool b_pos = pos_bits(B);  // B > 0, on the bits
    double first = b_pos ? (near_lo ? dlo : dhi) * rcp64(B) : 1.0;  // 1 - cos or 1 + cos (FP64)
    float f1 = d2f(first);
    float omc = b_pos ? (near_lo ? f1 : 2.0f - f1) : 1.0f;
    float opc = b_pos ? (near_lo ? 2.0f - f1 : f1) : 1.0f;
    float cth = (omc <= opc) ? 1.0f - omc : opc - 1.0f;
    float sth = sqrtf(fmaxf(omc * opc, 0.0f));
    float sph, cph;
    sincospif(2.0f * rphi, &sph, &cph);
    double m12 = m1 * m1, m22 = m2 * m2;
    float i2m0 = 0.5f / m0;
    float pabs = d2f(sqrt64(kallen64_m(s, m1, m2))) * i2m0;
    float e1 = d2f(s + m12 - m22) * i2m0, e2 = d2f(s + m22 - m12) * i2m0;
    float vx = pabs * sth * cph, vy = pabs * sth * sph, vz = pabs * cth;
    float rx = ca * vx + sa * vz, rz = -sa * vx + ca * vz;
    F4 q1 = {e1, cpa * rx - spa * vy, spa * rx + cpa * vy, rz};
    F4 q2 = {e2, -q1.x, -q1.y, -q1.z};
    p1 = boost_out(q1, p0, m0);
    p2 = boost_out(q2, p0, m0);
    return 0.5 * kPi * rcp64(sqrt64(kallen64(s, mA2, mB2)));
}

template <bool kBoost>
__device__ __forceinline__ double two_body(float rphi, float rth, double s0, double m1, double m2, F4 p0, F4& p1,
                                           F4& p2) {
    float sl, m0, i2m0, e1, e2;
    bool massless = zero_bits(m1) && zero_bits(m2);
    if (massless) {  // massless daughters: sqrt(lambda) = s0, E1 = E2 = s0/(2 m0)
        const float s0f = d2f(s0);
        sl = s0f;
        m0 = sqrtf(s0f);
        i2m0 = 0.5f / m0;
        e1 = e2 = s0f * i2m0;
    } else {
        double m12 = m1 * m1, m22 = m2 * m2;
        double lam = kallen64_m(s0, m1, m2);                   // FP64 island at threshold
        sl = sqrtf(d2f(lam));
        m0 = sqrtf(d2f(s0));
        i2m0 = 0.5f / m0;
        e1 = d2f(s0 + m12 - m22) * i2m0;
        e2 = d2f(s0 + m22 - m12) * i2m0;
    }
    float pabs = sl * i2m0;
    float cth = 2.0f * rth - 1.0f;
    float sth = 2.0f * sqrtf(rth * (1.0f - rth));
    float sph, cph;
    sincospif(2.0f * rphi, &sph, &cph);
    F4 q1 = {e1, pabs * sth * cph, pabs * sth * sph, pabs * cth};
    F4 q2 = {e2, -q1.x, -q1.y, -q1.z};
    if (kBoost) {
        p1 = boost_out(q1, p0, m0);
        p2 = boost_out(q2, p0, m0);
    } else {
        p1 = q1;
        p2 = q2;
    }
    // J = (pi/2) sqrt(lambda)/s0: pi/2 itself for massless daughters (NaN where s0 is not a
    // positive finite float, as the division would give), with no FP64 conversion
    if (massless) {
        const float s0f = d2f(s0);
        return (s0f > 0.0f && s0f <= 3.40282347e38f) ? f2d(0.5f * static_cast<float>(kPi))
                                              : __longlong_as_double(0x7FF8000000000000LL);
    }
    return f2d(0.5f * static_cast<float>(kPi) * sl / d2f(s0));
}

}  // namespace mx

// The register frame of a compiled mixed-precision channel: every slot has a double and a float
// register, and each write sets the one of its own type and the other's conversion (f2d, d2f).
// Reads take the register of the reader's type, so a value produced and consumed in the same
// precision is never converted, and a conversion nobody reads is dead code that the compiler
// drops: the conversions that remain are the edges of the FP64 islands, on the integer ALU.
template <int NS, class Imm>
struct MixRegFrame {
    static constexpr bool kStatic = true;
    mutable double v[NS > 0 ? NS : 1];
    mutable float w[NS > 0 ? NS : 1];
};
template <int NS, class Imm>
__device__ __forceinline__ double ld(const MixRegFrame<NS, Imm>& f, int a) { return a >= 0 ? f.v[a] : Imm::v(~a); }
template <int NS, class Imm>
__device__ __forceinline__ void st(const MixRegFrame<NS, Imm>& f, int slot, double x) {
    f.v[slot] = x;
    f.w[slot] = mx::d2f(x);
}
namespace mx {
template <int NS, class Imm>
__device__ __forceinline__ float ldf(const MixRegFrame<NS, Imm>& f, int a) { return a >= 0 ? f.w[a] : Imm::f(~a); }
// An op's float result enters later ops as a stored value, as it does from the shared-memory slot
// file: the empty asm keeps the compiler from contracting a product at the end of one op with a
// sum at the start of the next into one FMA (the interpreter rounds the product), so compiled
// and interpreted programs round the same way.
template <int NS, class Imm>
__device__ __forceinline__ void stf(const MixRegFrame<NS, Imm>& f, int slot, float x) {
    asm("" : "+f"(x));
    f.w[slot] = x;
    f.v[slot] = f2d(x);
}
template <int NS, class Imm>
__device__ __forceinline__ F4 ldp(const MixRegFrame<NS, Imm>& f, int a) { return {f.w[a], f.w[a + 1], f.w[a + 2], f.w[a + 3]}; }
template <int NS, class Imm>
__device__ __forceinline__ void stp(const MixRegFrame<NS, Imm>& f, int slot, F4 p) {
    stf(f, slot, p.e);
    stf(f, slot + 1, p.x);
    stf(f, slot + 2, p.y);
    stf(f, slot + 3, p.z);
}
}  // namespace mx


namespace mx {
// The FP32 form of sde_factor: the product as a float mantissa in [1, 2) and an integer exponent
// (no FP64 work per propagator); sde_weight turns it into P_j = 1/(acc 2^ex) once per channel.
__device__ __forceinline__ float sde_sq(const F4& q) { return fmaf(q.e, q.e, -fmaf(q.x, q.x, fmaf(q.y, q.y, q.z * q.z))); }
__device__ __forceinline__ void sde_factor_s(float& acc, int& ex, float s, int kind, float M, float G) {
    const float d = s - M * M, mg = M * G;
    acc *= (kind == 1) ? d * d : fmaf(d, d, mg * mg);
    const int bits = __float_as_int(acc);  // acc = 1.m 2^e with e moved into ex
    ex += ((bits >> 23) & 0xFF) - 127;
    acc = __int_as_float((bits & 0x807FFFFF) | 0x3F800000);
}
__device__ __forceinline__ void sde_factor(float& acc, int& ex, const F4& q, int kind, float M, float G) {
    sde_factor_s(acc, ex, sde_sq(q), kind, M, G);
}
// 1 / (acc 2^ex): the float 1/acc in (1/2, 1] widened to a double by its bits with -ex added
// to the exponent, on the integer ALU (|ex| stays far below 1000 here)
__device__ __forceinline__ double sde_weight(float acc, int ex) {
    const uint32_t u = __float_as_uint(1.0f / acc);
    return __hiloint2double(static_cast<int>((u >> 3) + 0x38000000u - (static_cast<uint32_t>(ex) << 20)),
                            static_cast<int>(u << 29));
}
}  // namespace mx

template <class Fr>
__device__ __forceinline__ void exec_op_mixed(const int op, const int32_t* a, const int32_t* o, const int na,
                                              const int no, const Fr& f, const float* gridf, int vbins,
                                              unsigned long long* cut_count, bool active) {
    using mx::F4;
        switch (op) {
            case PS_OP_VEGAS: {
                float jac = 1.0f;
                const float nb = static_cast<float>(vbins);
                op_loop<Fr>(0, na, 1, [&](int j) {
                    float r = mx::ldf(f, a[j]);
                    float rn = r * nb;
                    int k = max(min(static_cast<int>(rn), vbins - 1), 0);
                    const float e0 = gridf[j * (vbins + 1) + k];
                    const float wdt = gridf[na * (vbins + 1) + j * vbins + k];  // staged e[k+1] - e[k]
                    mx::stf(f, o[j], fmaf(rn - static_cast<float>(k), wdt, e0));
                    jac *= nb * wdt;
                });
                mx::stf(f, o[na], jac);
                break;
            }
            case PS_OP_INVARIANT_NU: {
                double x, j;
                mx::map_nu(mx::ldf(f, a[0]), ld(f, a[1]), ld(f, a[2]), ld(f, a[3]), ld(f, a[4]), ld(f, a[5]), x, j);
                st(f, o[0], x);
                st(f, o[1], j);
                break;
            }
            case PS_OP_INVARIANT_BW: {
                double x, j;
                mx::map_bw(mx::ldf(f, a[0]), ld(f, a[1]), ld(f, a[2]), ld(f, a[3]), ld(f, a[4]), x, j, na > 5,
                           na > 5 ? ld(f, a[5]) : 0.0);
                st(f, o[0], x);
                st(f, o[1], j);
                break;
            }
            case PS_OP_R_TO_X1X2: {
                float r = mx::ldf(f, a[0]);
                float S = mx::ldf(f, a[2]);
                float L = logf(mx::ldf(f, a[1]) / S);
                const float l1 = r * L, l2 = (1.0f - r) * L;  // log x1, log x2
                mx::stf(f, o[0], fminf(expf(l1), 1.0f));
                mx::stf(f, o[1], fminf(expf(l2), 1.0f));
                mx::stf(f, o[2], -L / S);
                if (no > 3) {
                    mx::stf(f, o[3], fminf(l1, 0.0f));
                    mx::stf(f, o[4], fminf(l2, 0.0f));
                }
                break;
            }
            case PS_OP_COM_P_IN: {
                float h = 0.5f * mx::ldf(f, a[0]);
                mx::stp(f, o[0], F4{h, 0.0f, 0.0f, h});
                mx::stp(f, o[1], F4{h, 0.0f, 0.0f, -h});
                break;
            }
            case PS_OP_T_INV_MIN_MAX: {
                double lo, hi, B;
                mx::t_range(ld(f, a[0]), ld(f, a[1]), ld(f, a[2]), ld(f, a[3]), ld(f, a[4]), lo, hi, B);
                st(f, o[0], lo);
                st(f, o[1], hi);
                break;
            }
            case PS_OP_TWO_TO_TWO_COM: {
                F4 p1, p2;
                double j = mx::two_to_two(mx::ldf(f, a[0]), mx::ldp(f, a[1]), mx::ldp(f, a[2]), ld(f, a[3]),
                                          ld(f, a[4]), ld(f, a[5]), ld(f, a[6]), ld(f, a[7]), ld(f, a[8]), p1, p2);
                mx::stp(f, o[0], p1);
                mx::stp(f, o[1], p2);
                st(f, o[2], j);
                break;
            }
            case PS_OP_TWO_BODY_DECAY: {
                F4 p1, p2;
                double j = mx::two_body<true>(mx::ldf(f, a[0]), mx::ldf(f, a[1]), ld(f, a[2]), ld(f, a[3]),
                                              ld(f, a[4]), mx::ldp(f, a[5]), p1, p2);
                mx::stp(f, o[0], p1);
                mx::stp(f, o[1], p2);
                st(f, o[2], j);
                break;
            }
            case PS_OP_TWO_BODY_DECAY_COM: {
                F4 p1, p2;
                double j = mx::two_body<false>(mx::ldf(f, a[0]), mx::ldf(f, a[1]), ld(f, a[2]), ld(f, a[3]),
                                               ld(f, a[4]), F4{0, 0, 0, 0}, p1, p2);
                mx::stp(f, o[0], p1);
                mx::stp(f, o[1], p2);
                st(f, o[2], j);
                break;
            }
            case PS_OP_BOOST_BEAM: {
                float x1 = mx::ldf(f, a[na - 2]), x2 = mx::ldf(f, a[na - 1]);
                float rho = sqrtf(x1 / x2);
                float irho = 1.0f / rho;
                op_loop<Fr>(0, na - 2, 1, [&](int k) {
                    F4 p = mx::ldp(f, a[k]);
                    float plus = rho * (p.e + p.z), minus = (p.e - p.z) * irho;
                    mx::stp(f, o[k], F4{0.5f * (plus + minus), p.x, p.y, 0.5f * (plus - minus)});
                });
                break;
            }
            case PS_OP_REDUCE_PRODUCT: {
                double v = ld(f, a[0]);
                op_loop<Fr>(1, na, 1, [&](int k) { v *= ld(f, a[k]); });
                st(f, o[0], v);
                break;
            }
            case PS_OP_CUT_UNPHYSICAL: {
                // x1, x2 are float values in the mixed form: a register frame tests them as floats
                // (no conversion), the shared-memory slot file on their FP64 bit patterns
                double w = ld(f, a[0]);
                bool xin;
                if constexpr (Fr::kStatic) {
                    const float x1 = mx::ldf(f, a[1]), x2 = mx::ldf(f, a[2]);
                    xin = x1 > 0.0f && x1 <= 1.0f && x2 > 0.0f && x2 <= 1.0f;
                } else {
                    xin = in_unit_bits(ld(f, a[1])) && in_unit_bits(ld(f, a[2]));
                }
                bool bad = !finite_bits(w) || !xin;
                op_loop<Fr>(3, na, 1, [&](int k) {
                    F4 p = mx::ldp(f, a[k]);
                    bad |= !(isfinite(p.e) && isfinite(p.x) && isfinite(p.y) && isfinite(p.z));
                });
                if (bad && active) atomicAdd(cut_count, 1ULL);
                st(f, o[0], bad ? 0.0 : w);
                break;
            }
            case PS_OP_ADD: st(f, o[0], ld(f, a[0]) + ld(f, a[1])); break;
            case PS_OP_SUB: st(f, o[0], ld(f, a[0]) - ld(f, a[1])); break;
            case PS_OP_MUL: st(f, o[0], ld(f, a[0]) * ld(f, a[1])); break;
            case PS_OP_DIV: st(f, o[0], ld(f, a[0]) / ld(f, a[1])); break;
            case PS_OP_SQRT: st(f, o[0], mx::sqrt64(ld(f, a[0]))); break;
            case PS_OP_SQUARE: { double v = ld(f, a[0]); st(f, o[0], v * v); break; }
            case PS_OP_MAX: st(f, o[0], fmax_bits(ld(f, a[0]), ld(f, a[1]))); break;
            case PS_OP_MOM_ADD: mx::stp(f, o[0], mx::f4_add(mx::ldp(f, a[0]), mx::ldp(f, a[1]))); break;
            case PS_OP_MOM_SUB: mx::stp(f, o[0], mx::f4_sub(mx::ldp(f, a[0]), mx::ldp(f, a[1]))); break;
            case PS_OP_PDF_POWER: {
                // x is a float value here (r_to_x1x2 of the mixed form), so 1 - x in float is the
                // correctly rounded difference, as the FP64 difference rounded to float would be;
                // the pair form as in the FP64 op
                const bool pair = na == 6;
                float x = mx::ldf(f, a[0]), al = mx::ldf(f, a[1]), be = mx::ldf(f, a[2]);
                float lx = na > 3 ? mx::ldf(f, a[3]) : logf(x);
                if (pair) lx = __fadd_rn(lx, mx::ldf(f, a[5]));
                float fx = expf(al * lx);
                auto pw = [&](float y) {
                    if (be == 3.0f) return y * y * y;
                    if (be == 2.0f) return y * y;
                    if (be == 1.0f) return y;
                    if (be == 0.0f) return 1.0f;
                    return powf(y, be);
                };
                float fy = pw(1.0f - x);
                if (pair) fy *= pw(1.0f - mx::ldf(f, a[4]));
                mx::stf(f, o[0], fx * fy);
                break;
            }
            case PS_OP_PROPAGATOR: {
                double M = ld(f, a[1]);
                float d = mx::d2f(ld(f, a[0]) - M * M);   // s - M^2 in FP64
                float mg = mx::d2f(M * ld(f, a[2]));
                mx::stf(f, o[0], 1.0f / (d * d + mg * mg));
                break;
            }
            case PS_OP_ONE_PLUS_COS2: {
                F4 p = mx::ldp(f, a[0]);
                float c2 = p.z * p.z / (p.x * p.x + p.y * p.y + p.z * p.z);
                mx::stf(f, o[0], 1.0f + c2);
                break;
            }
            case PS_OP_CHANNEL_WEIGHT: {
                // FP32 throughout, as the momenta it starts from: momentum sums, invariants and
                // denominators; the product of the denominators is kept as an FP32 mantissa in
                // [1, 2) and an integer exponent (no FP64 work per propagator), and P_j becomes a
                // double once per channel
                const int k = op_int<Fr>(ld(f, a[0]));
                const F4 pa = mx::ldp(f, a[1]);
                float acc = 1.0f;
                int ex = 0;
                op_loop<Fr>(2 + k, na - 3, 4, [&](int j) {
                    const int kind = op_int<Fr>(ld(f, a[j]));
                    const int mask = op_int<Fr>(ld(f, a[j + 1]));
                    const float M = mx::ldf(f, a[j + 2]), G = mx::ldf(f, a[j + 3]);
                    F4 q = (kind == 1) ? pa : F4{0.0f, 0.0f, 0.0f, 0.0f};
                    op_bits<Fr>(mask, k, [&](int i) {
                        q = (kind == 1) ? mx::f4_sub(q, mx::ldp(f, a[2 + i])) : mx::f4_add(q, mx::ldp(f, a[2 + i]));
                    });
                    mx::sde_factor(acc, ex, q, kind, M, G);
                });
                st(f, o[0], mx::sde_weight(acc, ex));
                break;
            }
            default: break;
        }
}

static __device__ void run_code_mixed(const int32_t* code, int len, const Frame& f, const float* gridf, int vbins,
                               unsigned long long* cut_count, bool active) {
    int pc = 0;
    while (pc < len) {
        const int op = code[pc], na = code[pc + 1], no = code[pc + 2];
        const int32_t* a = code + pc + 3;
        exec_op_mixed(op, a, a + na, na, no, f, gridf, vbins, cut_count, active);
        pc += 3 + na + no;
    }
}

// Locate the output descriptor [kOpOutput, n, 0, (role, slot)...] after the instructions.
__device__ __forceinline__ int find_output(const int32_t* code, int len) {
    int pc = 0;
    while (pc < len && code[pc] != kOpOutput) pc += 3 + code[pc + 1] + code[pc + 2];
    return pc;
}


// ---------------------------------------------------------------- event input and output
// Random inputs of one event into slots 0..n_random-1: explicit SoA, or Philox4x32-10 with
// counter (ev_lo, ev_hi, channel, j/2) and key (seed_lo, seed_hi).  Mixed-precision programs
// (kMix), whose maps read the random numbers as floats, take the float form of each coordinate
// directly from the bits (no FP64 work, no conversion).
template <bool kMix, class Fr>
__device__ __forceinline__ void load_inputs(const Fr& f, const LaunchParams& lp, int c, int n_random, int64_t ev,
                                            int64_t local, bool active) {
    if (lp.r != nullptr) {
        op_loop<Fr>(0, n_random, 1, [&](int j) { st(f, j, active ? lp.r[j * lp.ld_r + local] : 0.5); });
    } else {
        op_loop<Fr>(0, n_random, 2, [&](int j) {
            uint4 o = philox4x32_10(make_uint4(static_cast<uint32_t>(ev), static_cast<uint32_t>(ev >> 32),
                                               static_cast<uint32_t>(c), static_cast<uint32_t>(j >> 1)),
                                    static_cast<uint32_t>(lp.seed), static_cast<uint32_t>(lp.seed >> 32));
            if constexpr (kMix) {
                mx::stf(f, j, rng::unit_from_bits_f(o.y));
                if (j + 1 < n_random) mx::stf(f, j + 1, rng::unit_from_bits_f(o.w));
            } else {
                st(f, j, unit_from_bits(o.y, o.x));
                if (j + 1 < n_random) st(f, j + 1, unit_from_bits(o.w, o.z));
            }
        });
    }
}

// The declared outputs of one event (descriptor od = (role, slot) x n_out): FP64 programs write
// f64 everywhere, mixed programs momenta, x and alpha as f32.  Returns the weight.
template <bool kMix, class Fr>
__device__ __forceinline__ double store_outputs(const Fr& f, const int32_t* od, int n_out, const LaunchParams& lp,
                                                const ChannelLaunch& C, int64_t local, bool active) {
    double w = 0.0;
    int mom_k = 0;
    const int64_t col = C.col_off + local;
    op_loop<Fr>(0, n_out, 1, [&](int k) {
        const int role = od[2 * k], slot = od[2 * k + 1];
        if (role == PS_ROLE_MOMENTUM) {
            if (active && lp.mom != nullptr) {
                if constexpr (kMix) {
                    mx::F4 p = mx::ldp(f, slot);
                    float* m = static_cast<float*>(lp.mom) + static_cast<int64_t>(4 * mom_k) * lp.ld + col;
                    __stcs(m, p.e);
                    __stcs(m + lp.ld, p.x);
                    __stcs(m + 2 * lp.ld, p.y);
                    __stcs(m + 3 * lp.ld, p.z);
                } else {
                    P4 p = ldp(f, slot);
                    double* m = static_cast<double*>(lp.mom) + static_cast<int64_t>(4 * mom_k) * lp.ld + col;
                    __stcs(m, p.e);
                    __stcs(m + lp.ld, p.x);
                    __stcs(m + 2 * lp.ld, p.y);
                    __stcs(m + 3 * lp.ld, p.z);
                }
            }
            ++mom_k;
        } else {
            double v = ld(f, slot);
            if (role == PS_ROLE_WEIGHT) {
                w = v;
                if (active && lp.w != nullptr) __stcs(lp.w + col, v);
            } else {
                void* dst = role == PS_ROLE_X1 ? lp.x1 : role == PS_ROLE_X2 ? lp.x2 : lp.alpha;
                if (active && dst != nullptr) {
                    if constexpr (kMix) __stcs(static_cast<float*>(dst) + col, mx::ldf(f, slot));
                    else __stcs(static_cast<double*>(dst) + col, v);
                }
            }
        }
    });
    return w;
}

// ---------------------------------------------------------------- tile loop
// The persistent tile loop shared by the interpreter kernel and compiled kernels: tiles of
// `block` events over all channels (tile -> channel by the prefix sums in the parameters), a
// channel change stages the channel's shared data (pol.stage), every thread evaluates one event
// (pol.event -> weight), then the tile's partial sums.  (The VEGAS training histogram is a separate
// pass over the stored weights, in a fixed order.)
template <class Policy>
__device__ __forceinline__ void map_tiles(const LaunchParams& lp, Policy& pol, double* s_red) {
    const int B = lp.block;
    const int tid = threadIdx.x;
    int cur = -1;
    for (int64_t tile = blockIdx.x; tile < lp.n_tiles; tile += gridDim.x) {
        int c = 0;
        while (c + 1 < lp.n_ch && tile >= lp.ch[c + 1].tile_begin) ++c;
        const ChannelLaunch& C = lp.ch[c];
        if (c != cur) {
            __syncthreads();
            pol.stage(c, C);
            __syncthreads();
            cur = c;
        }
        const int64_t local = (tile - C.tile_begin) * B + tid;
        const bool active = local < C.n_events;
        const int64_t ev = C.ev_offset + local;
        double w = pol.event(c, C, ev, local, active);
        if (!active) w = 0.0;
        if (active && !finite_bits(w)) atomicAdd(lp.status + 0, 1ULL);

        // Per-tile partial statistics: nonzero count, sum w, sum w^2, max(0, max w).  The warp
        // stage spends six FP64 instructions per event: the count is a ballot, the maximum an
        // integer maximum of bit patterns (positive doubles order like their bits; NaN, negative
        // and zero weights enter as +0), and the two sums share one butterfly: at the first step
        // the lower half of the warp keeps sum w and the upper half sum w^2, each lane adding
        // the partner's copy of the one it keeps, and the remaining four steps run within
        // each half (lane 0 ends with sum w, lane 16 with sum w^2).
        const int warp = tid >> 5, lane = tid & 31;
        const unsigned full = 0xffffffffu;
        const int nz = __popc(__ballot_sync(full, (dbits(w) << 1) != 0));  // w != 0 (NaN counts)
        const double w2 = w * w;
        const bool upper = (lane & 16) != 0;
        double sum = upper ? w2 : w;
        sum += __shfl_xor_sync(full, upper ? w : w2, 16);
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) sum += __shfl_xor_sync(full, sum, off);
        const long long key = pos_bits(w) ? dbits(w) : 0LL;
        const unsigned kh = __reduce_max_sync(full, static_cast<unsigned>(key >> 32));
        const unsigned kl = __reduce_max_sync(full, static_cast<unsigned>(key >> 32) == kh
                                                        ? static_cast<unsigned>(key) : 0u);
        __syncthreads();  // s_red reuse across tiles
        if (lane == 0) {
            s_red[4 * warp + 0] = static_cast<double>(nz);
            s_red[4 * warp + 1] = sum;
            s_red[4 * warp + 3] = __longlong_as_double((static_cast<long long>(kh) << 32) | kl);
        } else if (lane == 16) {
            s_red[4 * warp + 2] = sum;
        }
        __syncthreads();
        if (tid == 0) {
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            for (int k = 0; k < B / 32; ++k) {
                a0 += s_red[4 * k];
                a1 += s_red[4 * k + 1];
                a2 += s_red[4 * k + 2];
                a3 = fmax(a3, s_red[4 * k + 3]);
            }
            double* tp = lp.tile_partials + 4 * tile;
            tp[0] = a0;
            tp[1] = a1;
            tp[2] = a2;
            tp[3] = a3;
        }
    }
}

// A compiled program's policy: the VEGAS grid is the only shared data; the generated `Events`
// evaluates channel c's instruction list on a register frame.
template <bool kMix, class Events>
struct CompiledPolicy {
    const LaunchParams& lp;
    double* s_grid;
    __device__ __forceinline__ void stage(int c, const ChannelLaunch& C) {
        double* g = s_grid + kTrigDoubles;  // after the azimuth table
        if constexpr (kMix) {
            stage_grid(reinterpret_cast<float*>(g), lp.grid + C.grid_off, C.vdims, C.vbins, threadIdx.x, lp.block);
        } else {
            stage_trig(s_grid, threadIdx.x, lp.block);
            stage_grid(g, lp.grid + C.grid_off, C.vdims, C.vbins, threadIdx.x, lp.block);
        }
    }
    __device__ __forceinline__ double event(int c, const ChannelLaunch& C, int64_t ev, int64_t local, bool active) {
        return Events::run(c, lp, C, ev, local, active, s_grid + kTrigDoubles, lp.status + 1);
    }
};

}  // namespace dev
}  // namespace ps
