/*
 * ps_oracle.c -- plain, slow FP64 CPU restatement of the phase-space hot path
 * of "MadSpace -- Event Generation for the Era of GPUs and ML" (arXiv 2602.06895).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product links, imports or calls this
 * file: only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * use it.  It shares no code, header, table or helper with the CUDA path.
 *
 * One event is processed at a time, in the order the paper gives the steps
 * (Sec. 2.2 building blocks, Sec. 2.2.7 s-channel order, Sec. 2.2.8 t-channel
 * order, Sec. 3.2 example compute graph).  All arithmetic is IEEE double,
 * compiled with -ffp-contract=off.  Transcendentals come from libm.
 *
 * Where the paper's literal formula cancels catastrophically at an edge of its
 * domain, an algebraically identical form is used instead; each such place says
 * which formula it restates and why (power-law map near x_min, Breit-Wigner near
 * u = +-pi/2, small |t|, Kallen function at threshold).
 *
 * Parity pins (tests/test_oracle_*.py) tie every function here to something the
 * paper or mathematics fixes: closed-form volumes, special cases, brute-force
 * finite-difference Jacobians, the inverse round trip and published Philox
 * known-answer vectors.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef __cplusplus  /* the operation-counting copy is compiled as C++ (op_count.h) */
extern "C" {
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_MAXN 32   /* topology nodes per channel */
#define ORC_MAXK 10   /* children per node (t-chain legs) */
#define ORC_MAXP 16   /* propagators per channel in the multichannel table */
#define ORC_MAXC 32   /* channels in the multichannel table */
#define ORC_NAUX 10
/* The condition numbers reported in aux[] (parity-test bookkeeping, not part of the method) are
 * computed unless a build sets ORC_BOOKKEEPING to 0, as the operation-counting build does. */
#ifndef ORC_BOOKKEEPING
#define ORC_BOOKKEEPING 1
#endif

/* ------------------------------------------------------------------------ */
/* Topology description (oracle-private layout; filled by oracle/__init__.py) */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t kind;            /* 0 = final-state leaf, 1 = s-channel 1->2 decay, 2 = t-chain (root only) */
    int32_t nchild;
    int32_t child[ORC_MAXK]; /* t-chain: legs ordered from incoming leg A to leg B */
    int32_t leaf;            /* leaf: output particle index */
    int32_t sde;             /* decay node: its propagator enters the channel's SDE product */
    double mass;             /* leaf: on-shell mass */
    double M, G, nu;         /* decay node: Breit-Wigner if G > 0, else power law with exponent nu around mass M */
} orc_node;

typedef struct {
    int32_t n;               /* final-state multiplicity */
    int32_t hadronic;        /* 1: PDF convolution (shat map + r_to_x1x2 + boost_beam); 0: fixed sqrt_s */
    int32_t n_nodes;
    int32_t n_sorder;
    int32_t sorder[ORC_MAXN];/* decay nodes (not the root) in s-invariant sampling order */
    int32_t tside[ORC_MAXK]; /* t-chain step i = 1..kappa-1: 0 = leg taken next to A, 1 = next to B */
    int32_t integrand;       /* 0 none, 1 (1 + cos^2 theta_1), 2 pdf x pdf x resonant props, 3 pdf x pdf x sum_c P_c, 4 same with alpha = 1/n_ch */
    int32_t vegas_dims, vegas_bins;
    int32_t partonic;        /* 1: leave the momenta in the partonic rest frame (no boost_beam) */
    double sqrt_s, S, a;     /* fixed energy; hadronic beam invariant; auxiliary shift m^2 = -a */
    double shat_M, shat_G, shat_nu;
    double t_nu, ts_nu;      /* exponent of the |t| map and of the t-chain invariants s_i */
    double Mt;               /* (unused by the map) */
    double pdf_a, pdf_b;     /* synthetic parton density f(x) = x^pdf_a (1-x)^pdf_b */
    orc_node node[ORC_MAXN];
} orc_channel;

typedef struct {
    int32_t kind;            /* 0: s = (sum_{i in mask} p_i)^2 ; 1: t = (p_a - sum_{i in mask} p_i)^2 */
    int32_t mask;
    double M, G;
} orc_prop;

typedef struct {
    int32_t n_ch;
    int32_t n_prop[ORC_MAXC];
    orc_prop prop[ORC_MAXC][ORC_MAXP];
} orc_sde;

/* ------------------------------------------------------------------------ */
/* Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)          */
/* ------------------------------------------------------------------------ */
/* The paper draws uniform random numbers inside its compute graph (Sec. 3.2)
 * but names no generator.  Philox4x32-10 from its published definition:
 * ten rounds of two 32x32->64 multiplies (M0 = 0xD2511F53, M1 = 0xCD9E8D57),
 * with the Weyl key schedule (W0 = 0x9E3779B9, W1 = 0xBB67AE85). */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 64 random bits -> double strictly inside (0,1): the top 52 bits k give
 * (k + 1/2) * 2^-52, exactly representable, in [2^-53, 1 - 2^-53]. */
double orc_bits_to_unit(uint64_t bits)
{
    uint64_t k = bits >> 12;
    return ((double)k + 0.5) * 0x1p-52;
}

/* Random point of event `ev` in channel `ch`: dimension j comes from Philox call
 * j/2 with counter (ev_lo, ev_hi, ch, j/2) and key (seed_lo, seed_hi); the even
 * dimension takes words (1,0) as (hi,lo), the odd one words (3,2). */
void orc_random_point(uint64_t seed, uint32_t ch, uint64_t ev, int d, double* r)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    for (int b = 0; 2 * b < d; ++b) {
        uint32_t ctr[4] = { (uint32_t)ev, (uint32_t)(ev >> 32), ch, (uint32_t)b };
        uint32_t o[4];
        orc_philox4x32_10(ctr, key, o);
        r[2 * b] = orc_bits_to_unit(((uint64_t)o[1] << 32) | o[0]);
        if (2 * b + 1 < d) r[2 * b + 1] = orc_bits_to_unit(((uint64_t)o[3] << 32) | o[2]);
    }
}

void orc_random_batch(uint64_t seed, uint32_t ch, uint64_t ev0, int64_t B, int d, double* r, int threads)
{
#pragma omp parallel for schedule(static) num_threads(threads)
    for (int64_t e = 0; e < B; ++e) orc_random_point(seed, ch, ev0 + (uint64_t)e, d, r + e * d);
}

/* ------------------------------------------------------------------------ */
/* Kinematic helpers                                                          */
/* ------------------------------------------------------------------------ */
/* Kallen function lambda(x,y,z) = (x-y-z)^2 - 4yz (Sec. 2.2.3), in a form without
 * cancellation for each sign pattern of y, z (x >= 0):
 *   y, z >= 0:  (x-(sqrt y+sqrt z)^2)(x-(sqrt y-sqrt z)^2)   (factorised; exact at threshold)
 *   y, z <= 0:  x^2 + 2x(|y|+|z|) + (|y|-|z|)^2              (sum of non-negative terms)
 *   otherwise:  (x-y-z)^2 - 4yz                             (-4yz >= 0)
 * The result is clamped at 0. */
double orc_kallen(double x, double y, double z)
{
    double l;
    if (y >= 0.0 && z >= 0.0) {
        double sy = sqrt(y), sz = sqrt(z);
        double p = sy + sz, m = sy - sz;
        l = (x - p * p) * (x - m * m);
    } else if (y <= 0.0 && z <= 0.0) {
        double Y = -y, Z = -z, d = Y - Z;
        l = x * x + 2.0 * x * (Y + Z) + d * d;
    } else {
        double u = x - y - z;
        l = u * u - 4.0 * y * z;
    }
    return l > 0.0 ? l : 0.0;
}

static double mdot(const double* p, const double* q) { return p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3]; }

/* Boost p, given in the rest frame of a momentum q of mass mq, into the frame in
 * which q = (q0, qvec): E' = (q0 E + q.p)/mq, p' = p + q [q.p/(mq (q0+mq)) + E/mq]. */
static void boost_from_rest(const double* p, const double* q, double mq, double* out)
{
    double qp = q[1] * p[1] + q[2] * p[2] + q[3] * p[3];
    double c = qp / (mq * (q[0] + mq)) + p[0] / mq;
    out[0] = (q[0] * p[0] + qp) / mq;
    out[1] = p[1] + q[1] * c;
    out[2] = p[2] + q[2] * c;
    out[3] = p[3] + q[3] * c;
}

/* Inverse of boost_from_rest: momentum p given in the frame of q -> rest frame of q. */
static void boost_to_rest(const double* p, const double* q, double mq, double* out)
{
    double qp = q[1] * p[1] + q[2] * p[2] + q[3] * p[3];
    double c = qp / (mq * (q[0] + mq)) - p[0] / mq;
    out[0] = (q[0] * p[0] - qp) / mq;
    out[1] = p[1] + q[1] * c;
    out[2] = p[2] + q[2] * c;
    out[3] = p[3] + q[3] * c;
}

/* Rotation R(phi,theta) = Rz(phi) Ry(theta) of Sec. 2.2.6, applied to v, with the
 * angles given by their cosines and sines. */
static void rotate(const double* v, double cth, double sth, double cph, double sph, double* o)
{
    double x = cth * v[0] + sth * v[2];
    double y = v[1];
    double z = -sth * v[0] + cth * v[2];
    o[0] = cph * x - sph * y;
    o[1] = sph * x + cph * y;
    o[2] = z;
}

/* Direction angles of a 3-vector n: cos/sin theta and cos/sin phi. */
static void direction(const double* n, double* cth, double* sth, double* cph, double* sph)
{
    double pt = sqrt(n[0] * n[0] + n[1] * n[1]);
    double pp = sqrt(pt * pt + n[2] * n[2]);
    *cth = n[2] / pp;
    *sth = pt / pp;
    if (pt > 0.0) { *cph = n[0] / pt; *sph = n[1] / pt; }
    else { *cph = 1.0; *sph = 0.0; }
}

/* ------------------------------------------------------------------------ */
/* Analytic invariant maps (Sec. 2.2.1)                                       */
/* ------------------------------------------------------------------------ */
/* Power-law map G_nu (Eq. prop_stable_nu) and its nu = 1 limit (Eq. prop_stable_nu1).
 * m <= 0 selects the auxiliary negative mass m^2 = -a.  With lo = x_min - m^2,
 * hi = x_max - m^2, L = log(hi/lo) = log1p((x_max - x_min)/lo) and w = 1 - nu, the paper's
 *     x = [r hi^w + (1-r) lo^w]^(1/w) + m^2,     1/g_nu = (hi^w - lo^w) (x - m^2)^nu / w
 * is the same as
 *   nu <= 1 (anchored at x_min):  z = r rho, rho = expm1(w L) >= 0,
 *        x = x_min + lo e,  e = expm1(log1p(z)/w),  J = lo (1+e) rho / (w (1+z))
 *   nu >  1 (anchored at x_max):  z = (1-r) rho', rho' = expm1(-w L) > 0,
 *        x - m^2 = hi exp(log1p(z)/w),  J = -(x - m^2) rho' / (w (1+z))
 * (hi^w = lo^w e^{wL}).  In either case 1 + z >= 1, so x - m^2 keeps full relative precision,
 * and for nu <= 1 also x - x_min.
 * nu = 1: x = x_min + lo expm1(r L), J = lo (1 + expm1(r L)) L.
 * Returns 0 on success, 1 if x_min - m^2 <= 0 or x_max < x_min (x = x_min, J = 0). */
int orc_map_nu(double r, double m, double nu, double xmin, double xmax, double a, double* x, double* jac)
{
    double m2 = (m > 0.0) ? m * m : -a;
    double lo = xmin - m2, hi = xmax - m2;
    if (!(lo > 0.0) || !(hi >= lo)) { *x = xmin; *jac = 0.0; return 1; }
    double L = log1p((xmax - xmin) / lo);
    if (nu == 1.0) {
        double e = expm1(r * L);
        *x = xmin + lo * e;
        *jac = (lo + lo * e) * L;
    } else if (nu < 1.0) {
        double w = 1.0 - nu;
        double rho = expm1(w * L);
        double z = r * rho;
        double e = expm1(log1p(z) / w);
        *x = xmin + lo * e;
        *jac = (lo + lo * e) * rho / (w * (1.0 + z));
    } else {
        double w = 1.0 - nu;
        double rho = expm1(-w * L);
        double z = (1.0 - r) * rho;
        double xm = hi * exp(log1p(z) / w); /* x - m^2 */
        *x = m2 + xm;
        *jac = -xm * rho / (w * (1.0 + z));
    }
    *x = fmin(fmax(*x, xmin), xmax); /* G maps into [x_min, x_max] (rounding at the ends) */
    return 0;
}

/* Inverse of orc_map_nu: r from x. */
double orc_inv_nu(double x, double m, double nu, double xmin, double xmax, double a)
{
    double m2 = (m > 0.0) ? m * m : -a;
    double lo = xmin - m2, hi = xmax - m2;
    double L = log1p((xmax - xmin) / lo);
    if (nu == 1.0) return log1p((x - xmin) / lo) / L;
    double w = 1.0 - nu;
    if (nu < 1.0) return expm1(w * log1p((x - xmin) / lo)) / expm1(w * L);
    return 1.0 - expm1(w * log((x - m2) / hi)) / expm1(-w * L);
}

/* Breit-Wigner map G_BW (Eq. prop_massive): x = m^2 + m Gamma tan(u1 + (u2-u1) r),
 * u_{1,2} = atan((x_{min,max} - m^2)/(m Gamma)), and 1/g_BW = (u2-u1) m Gamma (1 + tan^2 u).
 * With a = tan u1, b = tan u2, D = u2 - u1 = atan2(b - a, 1 + a b) (angle difference, exact
 * also for narrow ranges) and u = u1 + D r:
 *   u < -pi/4:  T = tan(D r),     x = x_min + m Gamma T (1+a^2)/(1 - aT),
 *               1 + tan^2 u = (1+a^2)(1+T^2)/(1-aT)^2          (angle addition from u1)
 *   u >  pi/4:  T = tan(D (1-r)), tan u = (b-T)/(1+bT), x = m^2 + m Gamma tan u,
 *               1 + tan^2 u = (1+b^2)(1+T^2)/(1+bT)^2          (angle subtraction from u2)
 *   otherwise:  x = m^2 + m Gamma tan u.
 * The edge branches avoid tan near +-pi/2; below the peak x is measured from x_min, which also
 * avoids the cancellation of m^2 + m Gamma tan u as x -> x_min. */
int orc_map_bw(double r, double M, double G, double xmin, double xmax, double* x, double* jac)
{
    double mg = M * G, m2 = M * M;
    if (!(mg > 0.0) || !(xmax >= xmin)) { *x = xmin; *jac = 0.0; return 1; }
    double a = (xmin - m2) / mg, b = (xmax - m2) / mg;
    double D = atan2((xmax - xmin) / mg, 1.0 + a * b);
    double u = atan(a) + D * r;
    if (u < -ORC_PI / 4) {
        double T = tan(D * r);
        double den = 1.0 - a * T;
        *x = xmin + mg * (T * (1.0 + a * a) / den);
        *jac = D * mg * ((1.0 + a * a) * (1.0 + T * T) / (den * den));
    } else if (u > ORC_PI / 4) {
        double T = tan(D * (1.0 - r));
        double den = 1.0 + b * T;
        *x = m2 + mg * ((b - T) / den);
        *jac = D * mg * ((1.0 + b * b) * (1.0 + T * T) / (den * den));
    } else {
        double t = tan(u);
        *x = m2 + mg * t;
        *jac = D * mg * (1.0 + t * t);
    }
    *x = fmin(fmax(*x, xmin), xmax); /* G maps into [x_min, x_max] (rounding at the ends) */
    return 0;
}

/* Inverse of orc_map_bw: the angle from the nearer endpoint,
 * u - u1 = atan2(x - x_min, m Gamma (1 + a t)) and u2 - u = atan2(x_max - x, m Gamma (1 + b t)),
 * with t = (x - m^2)/(m Gamma). */
double orc_inv_bw(double x, double M, double G, double xmin, double xmax)
{
    double mg = M * G, m2 = M * M;
    double a = (xmin - m2) / mg, b = (xmax - m2) / mg;
    double D = atan2((xmax - xmin) / mg, 1.0 + a * b);
    double t = (x - m2) / mg;
    if (x - xmin <= xmax - x) return atan2((x - xmin) / mg, 1.0 + a * t) / D;
    return 1.0 - atan2((xmax - x) / mg, 1.0 + b * t) / D;
}

/* PDF convolution (Sec. 2.2.2, Eq. pdf_sampling): tau = shat/S, x1 = tau^r,
 * x2 = tau^(1-r), and dx1 dx2 = dshat/S * |log tau| dr, i.e. J = -log(tau)/S. */
void orc_r_to_x1x2(double r, double shat, double S, double* x1, double* x2, double* jac)
{
    double L = log(shat / S);
    *x1 = exp(r * L);
    *x2 = exp((1.0 - r) * L);
    *jac = -L / S;
}

/* ------------------------------------------------------------------------ */
/* Two-particle blocks                                                        */
/* ------------------------------------------------------------------------ */
/* 1->2 decay in (phi, theta) (Sec. 2.2.3, Eq. ps2_phi_theta).  Parent invariant s0,
 * daughter masses m1, m2; phi = 2 pi r_phi, cos theta = 2 r_theta - 1.  Momenta are
 * built in the parent rest frame (sin theta = 2 sqrt(r_theta (1-r_theta))) and, if
 * p0 != NULL, boosted to the frame of p0 by a pure boost.  Returns the Jacobian
 * 4 pi * sqrt(lambda)/(8 s0) = pi sqrt(lambda)/(2 s0). */
double orc_two_body_decay(double rphi, double rth, double s0, double m1, double m2,
                          const double* p0, double* p1, double* p2)
{
    double m0 = sqrt(s0);
    double lam = orc_kallen(s0, m1 * m1, m2 * m2);
    double sl = sqrt(lam);
    double pabs = sl / (2.0 * m0);
    double e1 = (s0 + m1 * m1 - m2 * m2) / (2.0 * m0);
    double e2 = (s0 + m2 * m2 - m1 * m1) / (2.0 * m0);
    double cth = 2.0 * rth - 1.0;
    double sth = 2.0 * sqrt(rth * (1.0 - rth));
    double phi = 2.0 * ORC_PI * rphi;
    double cph = cos(phi), sph = sin(phi);
    double q1[4] = { e1, pabs * sth * cph, pabs * sth * sph, pabs * cth };
    double q2[4] = { e2, -q1[1], -q1[2], -q1[3] };
    if (p0) { boost_from_rest(q1, p0, m0, p1); boost_from_rest(q2, p0, m0, p2); }
    else { memcpy(p1, q1, sizeof q1); memcpy(p2, q2, sizeof q2); }
    return ORC_PI * sl / (2.0 * s0);
}

/* t-range of a 2->2 block (Sec. 2.2.4, Eq. t_invariant_theta): t = A + B cos theta with
 *   A = mA^2 + m1^2 - (s + mA^2 - mB^2)(s + m1^2 - m2^2)/(2s),  B = sqrt(L_AB L_12)/(2s).
 * |t| lies in [-(A+B), -(A-B)].  The root of larger magnitude is taken directly, the other
 * from the product of the roots, which expands to
 *   t+ t- = (m1^2 - mA^2)(m2^2 - mB^2) + (m1^2 mB^2 - m2^2 mA^2)(m1^2 - m2^2 - mA^2 + mB^2)/s
 * (exact zero for massless legs, where the direct difference cancels). */
void orc_t_min_max(double s, double mA2, double mB2, double m1, double m2, double* tabs_min, double* tabs_max)
{
    double m12 = m1 * m1, m22 = m2 * m2;
    double A = mA2 + m12 - (s + mA2 - mB2) * (s + m12 - m22) / (2.0 * s);
    double B = sqrt(orc_kallen(s, mA2, mB2) * orc_kallen(s, m12, m22)) / (2.0 * s);
    double P = (m12 - mA2) * (m22 - mB2) + (m12 * mB2 - m22 * mA2) * (m12 - m22 - mA2 + mB2) / s;
    double tplus, tminus; /* t+ = A + B (closest to 0), t- = A - B */
    if (A <= 0.0) { tminus = A - B; tplus = (tminus != 0.0) ? P / tminus : 0.0; }
    else { tplus = A + B; tminus = P / tplus; }
    *tabs_min = -tplus;
    *tabs_max = -tminus;
}

/* 2->2 block in (phi, t) (Sec. 2.2.4, Eqs. t_invariant_theta, 2_to_2_mapping, ps2_phi_t).
 * pA, pB: incoming momenta of the block, s = (pA+pB)^2, mA2/mB2 their invariant masses.
 * In the rest frame of p0 = pA + pB the polar axis is the direction of pA; cos theta follows
 * from |t| through 1 - cos theta = (|t| - |t|_min)/B (resp. 1 + cos theta = (|t|_max - |t|)/B),
 * phi = 2 pi r_phi; p1 is rotated by R(phi_A, theta_A) (Sec. 2.2.6) and both outgoing
 * momenta are boosted back.  Returns 2 pi/(4 sqrt(lambda(s, mA^2, mB^2))). */
double orc_two_to_two(double rphi, const double* pA, const double* pB, double tabs,
                      double m1, double m2, double s, double mA2, double mB2, double* p1, double* p2)
{
    double p0[4] = { pA[0] + pB[0], pA[1] + pB[1], pA[2] + pB[2], pA[3] + pB[3] };
    double m0 = sqrt(s);
    double pAs[4];
    boost_to_rest(pA, p0, m0, pAs);
    double cA, sA, cpA, spA;
    direction(pAs + 1, &cA, &sA, &cpA, &spA);

    double m12 = m1 * m1, m22 = m2 * m2;
    double tmin, tmax;
    orc_t_min_max(s, mA2, mB2, m1, m2, &tmin, &tmax);
    double B = sqrt(orc_kallen(s, mA2, mB2) * orc_kallen(s, m12, m22)) / (2.0 * s);
    double omc, opc; /* 1 - cos theta, 1 + cos theta */
    if (B > 0.0) {
        if (tabs - tmin <= tmax - tabs) { omc = (tabs - tmin) / B; opc = 2.0 - omc; }
        else { opc = (tmax - tabs) / B; omc = 2.0 - opc; }
    } else { omc = 1.0; opc = 1.0; }
    double cth = (omc <= opc) ? 1.0 - omc : opc - 1.0;
    double sth2 = omc * opc;
    double sth = sqrt(sth2 > 0.0 ? sth2 : 0.0);
    double phi = 2.0 * ORC_PI * rphi;
    double cph = cos(phi), sph = sin(phi);
    double pabs = sqrt(orc_kallen(s, m12, m22)) / (2.0 * m0);
    double e1 = (s + m12 - m22) / (2.0 * m0);
    double e2 = (s + m22 - m12) / (2.0 * m0);
    double v[3] = { pabs * sth * cph, pabs * sth * sph, pabs * cth };
    double q1[4], q2[4];
    q1[0] = e1;
    rotate(v, cA, sA, cpA, spA, q1 + 1);
    q2[0] = e2; q2[1] = -q1[1]; q2[2] = -q1[2]; q2[3] = -q1[3];
    boost_from_rest(q1, p0, m0, p1);
    boost_from_rest(q2, p0, m0, p2);
    return 2.0 * ORC_PI / (4.0 * sqrt(orc_kallen(s, mA2, mB2)));
}

/* Longitudinal boost from the partonic rest frame to the lab (boost_beam, Sec. 3.2) with
 * beta = (x1-x2)/(x1+x2), gamma = (x1+x2)/(2 sqrt(x1 x2)), written on the light cone:
 * E' + p_z' = rho (E + p_z), E' - p_z' = (E - p_z)/rho, rho = sqrt(x1/x2).  The same boost
 * without the cancellation of gamma E + gamma beta p_z for extreme boosts (the incoming
 * partons come out as exactly x_i sqrt(S)/2). */
static void boost_beam(double* p, double x1, double x2)
{
    double rho = sqrt(x1 / x2);
    double plus = rho * (p[0] + p[3]);
    double minus = (p[0] - p[3]) / rho;
    p[0] = 0.5 * (plus + minus);
    p[3] = 0.5 * (plus - minus);
}

static void unboost_beam(double* p, double x1, double x2)
{
    double rho = sqrt(x1 / x2);
    double plus = (p[0] + p[3]) / rho;
    double minus = rho * (p[0] - p[3]);
    p[0] = 0.5 * (plus + minus);
    p[3] = 0.5 * (plus - minus);
}

/* ------------------------------------------------------------------------ */
/* VEGAS grid (Lepage 1978): lookup, inverse, histogram, rebinning            */
/* ------------------------------------------------------------------------ */
/* Piecewise-linear map of one dimension through bin edges e[0..N]:
 * k = min(floor(r N), N-1), delta = r N - k, r' = e_k + delta (e_{k+1}-e_k),
 * Jacobian N (e_{k+1} - e_k). */
double orc_vegas_map(double r, const double* e, int N, double* jac)
{
    double rn = r * (double)N;
    int k = (int)floor(rn);
    if (k > N - 1) k = N - 1;
    if (k < 0) k = 0;
    double delta = rn - (double)k;
    double w = e[k + 1] - e[k];
    *jac *= (double)N * w;
    return e[k] + delta * w;
}

double orc_vegas_inv(double rp, const double* e, int N)
{
    int lo = 0, hi = N; /* find k with e[k] <= rp < e[k+1] */
    while (hi - lo > 1) { int mid = (lo + hi) / 2; if (e[mid] <= rp) lo = mid; else hi = mid; }
    double w = e[lo + 1] - e[lo];
    double delta = (rp - e[lo]) / w;
    return ((double)lo + delta) / (double)N;
}

/* Accumulate the VEGAS importance histogram: for every event and mapped dimension j,
 * hist[j][k_j] += w^2, with k_j the bin of the (unmapped) random number r_j. */
void orc_vegas_accumulate(const double* r, int d, const double* w, int64_t B, int dv, int N, double* hist)
{
    for (int64_t e = 0; e < B; ++e) {
        double w2 = w[e] * w[e];
        for (int j = 0; j < dv; ++j) {
            int k = (int)floor(r[e * d + j] * (double)N);
            if (k > N - 1) k = N - 1;
            hist[j * N + k] += w2;
        }
    }
}

/* Lepage's rebinning of one dimension: 3-point smoothing of the bin importances,
 * normalisation, compression m_k = ((1 - d_k)/log(1/d_k))^alpha, then new edges that
 * give every new bin an equal share of sum m_k (linear inside old bins). */
void orc_vegas_rebin(const double* hist, const double* e_old, double* e_new, int N, double alpha)
{
    double* d = (double*)malloc(sizeof(double) * N);
    double* m = (double*)malloc(sizeof(double) * N);
    double tot = 0.0;
    for (int k = 0; k < N; ++k) {
        double s;
        if (N == 1) s = hist[0];
        else if (k == 0) s = (hist[0] + hist[1]) / 2.0;
        else if (k == N - 1) s = (hist[N - 2] + hist[N - 1]) / 2.0;
        else s = (hist[k - 1] + hist[k] + hist[k + 1]) / 3.0;
        d[k] = s;
        tot += s;
    }
    if (!(tot > 0.0)) { memcpy(e_new, e_old, sizeof(double) * (N + 1)); free(d); free(m); return; }
    double msum = 0.0;
    for (int k = 0; k < N; ++k) {
        double dk = d[k] / tot;
        double mk = 0.0;
        if (dk >= 1.0) mk = 1.0;
        else if (dk > 0.0) mk = pow((1.0 - dk) / log(1.0 / dk), alpha);
        m[k] = mk;
        msum += mk;
    }
    double step = msum / (double)N;
    e_new[0] = e_old[0];
    e_new[N] = e_old[N];
    int k = 0;
    double acc = 0.0; /* sum of m over old bins before bin k */
    for (int j = 1; j < N; ++j) {
        double target = step * (double)j;
        while (k < N - 1 && acc + m[k] < target) { acc += m[k]; ++k; }
        double frac = (m[k] > 0.0) ? (target - acc) / m[k] : 0.0;
        if (frac > 1.0) frac = 1.0;
        if (frac < 0.0) frac = 0.0;
        e_new[j] = e_old[k] + frac * (e_old[k + 1] - e_old[k]);
    }
    free(d);
    free(m);
}

/* ------------------------------------------------------------------------ */
/* Channel map: recursive decomposition (Sec. 2.2, Eq. ps_decomposition)     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int parent[ORC_MAXN];
    int d_shat, d_x;
    int d_s[ORC_MAXN];                       /* decay node -> invariant dimension */
    int d_ts[ORC_MAXK];                      /* t-chain invariant s_i, i = 1..kappa-1 */
    int d_tphi[ORC_MAXK + 1], d_tt[ORC_MAXK + 1]; /* t-block i = 1..kappa */
    int d_dphi[ORC_MAXN], d_dth[ORC_MAXN];   /* decay node angles */
    int preorder[ORC_MAXN];
    int n_pre;
    int d;
} layout;

static void preorder_walk(const orc_channel* ch, int j, layout* L)
{
    const orc_node* nd = &ch->node[j];
    if (nd->kind == 1) L->preorder[L->n_pre++] = j;
    for (int k = 0; k < nd->nchild; ++k) preorder_walk(ch, nd->child[k], L);
}

/* Random-dimension order (generalising the example graph of Sec. 3.2): shat, the
 * s-channel invariants in sampling order, the t-chain invariants, x1x2, then (r_phi, r_t)
 * for every t-block, then (r_phi, r_theta) for every decay in pre-order. */
static int make_layout(const orc_channel* ch, layout* L)
{
    memset(L, -1, sizeof *L);
    for (int j = 0; j < ch->n_nodes; ++j)
        for (int k = 0; k < ch->node[j].nchild; ++k) L->parent[ch->node[j].child[k]] = j;
    int idx = 0;
    if (ch->hadronic) L->d_shat = idx++;
    for (int i = 0; i < ch->n_sorder; ++i) L->d_s[ch->sorder[i]] = idx++;
    int kappa = (ch->node[0].kind == 2) ? ch->node[0].nchild - 1 : 0;
    for (int i = 1; i < kappa; ++i) L->d_ts[i] = idx++;
    if (ch->hadronic) L->d_x = idx++;
    for (int i = 1; i <= kappa; ++i) { L->d_tphi[i] = idx++; L->d_tt[i] = idx++; }
    L->n_pre = 0;
    preorder_walk(ch, 0, L);
    for (int i = 0; i < L->n_pre; ++i) { L->d_dphi[L->preorder[i]] = idx++; L->d_dth[L->preorder[i]] = idx++; }
    L->d = idx;
    return idx;
}

int orc_channel_dims(const orc_channel* ch)
{
    layout L;
    return make_layout(ch, &L);
}

/* Minimal mass of a node (Sec. 2.2.7 step 2): leaf mass, sqrt(s_j) once sampled,
 * else the sum over children. */
static double min_mass(const orc_channel* ch, int j, const int* sampled, const double* s)
{
    const orc_node* nd = &ch->node[j];
    if (nd->kind == 0) return nd->mass;
    if (sampled[j]) return sqrt(s[j]);
    double m = 0.0;
    for (int k = 0; k < nd->nchild; ++k) m += min_mass(ch, nd->child[k], sampled, s);
    return m;
}

/* Maximal mass of node i (Sec. 2.2.7 step 3): walk towards the root until a sampled
 * node r; subtract the minimal masses of every node branching off the path. */
static double max_mass(const orc_channel* ch, const layout* L, int i, const int* sampled, const double* s,
                       double* subtracted)
{
    double sum = 0.0;
    int cur = i;
    for (;;) {
        int p = L->parent[cur];
        const orc_node* pn = &ch->node[p];
        for (int k = 0; k < pn->nchild; ++k)
            if (pn->child[k] != cur) sum += min_mass(ch, pn->child[k], sampled, s);
        if (sampled[p]) {
            if (subtracted) *subtracted = sum;
            return sqrt(s[p]) - sum;
        }
        cur = p;
    }
}

static double leg_mass(const orc_channel* ch, int j, const double* s)
{
    return ch->node[j].kind == 0 ? ch->node[j].mass : sqrt(s[j]);
}

static double prop_factor(double s, double M, double G)
{
    double d = s - M * M;
    return 1.0 / (d * d + M * M * G * G);
}

static double pdf(const orc_channel* ch, double x) { return pow(x, ch->pdf_a) * pow(1.0 - x, ch->pdf_b); }

/* Channel weight P_j of the SDE multichannel weights (Sec. 2.1, "products of propagator
 * denominators"), evaluated from lab-frame momenta; mom = [p_a, p_b, p_1..p_n]. */
static double sde_from_momenta(const orc_sde* sde, int j, const double* mom)
{
    double P = 1.0;
    for (int k = 0; k < sde->n_prop[j]; ++k) {
        const orc_prop* pr = &sde->prop[j][k];
        double q[4] = { 0, 0, 0, 0 };
        if (pr->kind == 1) { for (int mu = 0; mu < 4; ++mu) q[mu] = mom[mu]; }
        for (int i = 0; i < 30; ++i)
            if (pr->mask & (1 << i)) {
                double sg = (pr->kind == 1) ? -1.0 : 1.0;
                for (int mu = 0; mu < 4; ++mu) q[mu] += sg * mom[(2 + i) * 4 + mu];
            }
        double inv = mdot(q, q);
        if (pr->kind == 1) { double d = inv - pr->M * pr->M; P *= 1.0 / (d * d); }
        else P *= prop_factor(inv, pr->M, pr->G);
    }
    return P;
}

/* aux outputs per event */
enum { AUX_SHAT = 0, AUX_WPS, AUX_F, AUX_JV, AUX_POWN, AUX_CUT, AUX_FAIL, AUX_SPARE, AUX_COND, AUX_CONDP };

/* Forward map of one event.  r: d random numbers in (0,1).  mom: (n+2)*4 lab momenta
 * [p_a, p_b, p_1..p_n]; x[2]: x1, x2 (1, 1 at fixed energy); returns the weight. */
static double forward_event(const orc_channel* ch, const orc_sde* sde, int chan, const double* grid,
                            const double* r_in, double* mom, double* x, double* alpha_out, double* aux)
{
    layout L;
    make_layout(ch, &L);
    double r[64];
    memcpy(r, r_in, sizeof(double) * L.d);
    const int n = ch->n;
    int fail = 0;

    /* VEGAS on the first vegas_dims dimensions (Sec. 3.2.2) */
    double jv = 1.0;
    for (int j = 0; j < ch->vegas_dims; ++j)
        r[j] = orc_vegas_map(r[j], grid + j * (ch->vegas_bins + 1), ch->vegas_bins, &jv);

    double jac = pow(2.0 * ORC_PI, 4 - 3 * n) * jv; /* (2 pi)^(4-3n), Sec. 2.2 */
    double cond = 1.0;  /* weight: largest condition number of a range width, threshold or x factor */
    double condp = 1.0; /* momenta: rounding amplification -- threshold and backward-t condition numbers
                         * (both propagate through the later legs of a t-chain), gamma^2 of boosts into
                         * rest frames of composite momenta */
    double s[ORC_MAXN];
    int sampled[ORC_MAXN];
    memset(sampled, 0, sizeof sampled);
    for (int j = 0; j < ORC_MAXN; ++j) s[j] = 0.0;

    /* shat (Sec. 2.2.2): BW if the channel says so, else power law (nu ~ 1) */
    double shat, j1;
    if (ch->hadronic) {
        double smin = 0.0;
        for (int j = 0; j < ch->n_nodes; ++j) if (ch->node[j].kind == 0) smin += ch->node[j].mass;
        smin = smin * smin;
        if (ch->shat_G > 0.0) fail |= orc_map_bw(r[L.d_shat], ch->shat_M, ch->shat_G, smin, ch->S, &shat, &j1);
        else fail |= orc_map_nu(r[L.d_shat], ch->shat_M, ch->shat_nu, smin, ch->S, ch->a, &shat, &j1);
        jac *= j1;
    } else {
        shat = ch->sqrt_s * ch->sqrt_s;
    }
    s[0] = shat;
    sampled[0] = 1;

    /* s-channel invariants in the given order with recursive bounds (Sec. 2.2.7) */
    double P_own = 1.0;
    for (int i = 0; i < ch->n_sorder; ++i) {
        int j = ch->sorder[i];
        const orc_node* nd = &ch->node[j];
        double mlo = min_mass(ch, j, sampled, s);
        double max_mass_sub = 0.0;
        double mhi = max_mass(ch, &L, j, sampled, s, &max_mass_sub);
        double smin = mlo * mlo, smax = mhi > 0.0 ? mhi * mhi : 0.0;
        if (mhi < mlo) { fail = 1; smax = smin; }
        /* condition number of the range width: sqrt(s_r) / (m_max - m_min), with sqrt(s_r) = m_max + (the
         * masses subtracted); a rounding of the masses is amplified by it in the width */
        if (ORC_BOOKKEEPING) {
            double top = mhi + (max_mass_sub);
            double wdt = mhi - mlo;
            double k = wdt > 0.0 ? top / wdt : 1e300;
            if (k > cond) cond = k;
        }
        double sv;
        if (nd->G > 0.0) fail |= orc_map_bw(r[L.d_s[j]], nd->M, nd->G, smin, smax, &sv, &j1);
        else fail |= orc_map_nu(r[L.d_s[j]], nd->M, nd->nu, smin, smax, ch->a, &sv, &j1);
        jac *= j1;
        s[j] = sv;
        sampled[j] = 1;
        if (nd->sde) {
            P_own *= prop_factor(sv, nd->M, nd->G);
            if (ORC_BOOKKEEPING) {
                /* a propagator near a narrow peak amplifies an ulp of s by 2 s |s-M^2| / ((s-M^2)^2 + M^2 G^2) */
                double dd = sv - nd->M * nd->M;
                double k = 2.0 * sv * fabs(dd) / (dd * dd + nd->M * nd->M * nd->G * nd->G);
                if (k > cond) cond = k;
            }
        }
    }

    /* t-chain invariants s_1..s_{kappa-1} (Sec. 2.2.8): legs are taken inwards from
     * side A or B; s_i is the mass^2 of the legs not yet taken. */
    const orc_node* root = &ch->node[0];
    int kappa = (root->kind == 2) ? root->nchild - 1 : 0;
    int order[ORC_MAXK + 1];   /* sigma(1..kappa+1) as indices into root->child */
    int sideof[ORC_MAXK + 1];  /* 0 = A, 1 = B for steps 1..kappa-1 */
    double sts[ORC_MAXK + 1];
    if (kappa > 0) {
        int left = 0, right = kappa;
        for (int i = 1; i < kappa; ++i) {
            if (ch->tside[i] == 0) { order[i] = left++; sideof[i] = 0; }
            else { order[i] = right--; sideof[i] = 1; }
        }
        order[kappa] = left;
        order[kappa + 1] = right;
        sts[0] = shat;
        for (int i = 1; i < kappa; ++i) {
            double msum = 0.0;
            /* remaining legs after removing sigma(1..i) */
            int l2 = 0, r2 = kappa;
            for (int k = 1; k <= i; ++k) { if (sideof[k] == 0) ++l2; else --r2; }
            for (int k = l2; k <= r2; ++k) msum += leg_mass(ch, root->child[k], s);
            double mi = leg_mass(ch, root->child[order[i]], s);
            double smin = msum * msum;
            double mx = sqrt(sts[i - 1]) - mi;
            double smax = mx > 0.0 ? mx * mx : 0.0;
            if (smax < smin) { fail = 1; smax = smin; }
            if (ORC_BOOKKEEPING) {
                double wdt = mx - msum;
                double k = wdt > 0.0 ? sqrt(sts[i - 1]) / wdt : 1e300;
                if (k > cond) cond = k;
            }
            double sv;
            fail |= orc_map_nu(r[L.d_ts[i]], 0.0, ch->ts_nu, smin, smax, ch->a, &sv, &j1);
            jac *= j1;
            sts[i] = sv;
        }
    }

    /* x1, x2 (Sec. 2.2.2) */
    double x1 = 1.0, x2 = 1.0;
    if (ch->hadronic) {
        orc_r_to_x1x2(r[L.d_x], shat, ch->S, &x1, &x2, &j1);
        jac *= j1;
        if (ORC_BOOKKEEPING) {
            /* J_x = -log(tau)/S: shat carries up to ~30 ulps (an exponential of an argument up to
             * log(S/a)), which 1/|log tau| amplifies as tau -> 1 */
            double k = 30.0 / fabs(log(shat / ch->S));
            if (k > cond) cond = k;
        }
    }

    /* incoming partons in the partonic rest frame (com_p_in) */
    double p[ORC_MAXN][4];
    double rs = sqrt(shat);
    double pa[4] = { rs / 2, 0, 0, rs / 2 }, pb[4] = { rs / 2, 0, 0, -rs / 2 };
    double own_t_props = 1.0;

    if (kappa > 0) {
        double pA[4], pB[4];
        memcpy(pA, pa, sizeof pA);
        memcpy(pB, pb, sizeof pB);
        double mA2 = 0.0, mB2 = 0.0, scur = shat;
        for (int i = 1; i <= kappa; ++i) {
            double mt1, mt2;
            int leg1, leg2 = -1;
            if (i == kappa) {
                leg1 = root->child[order[kappa]];
                leg2 = root->child[order[kappa + 1]];
                mt1 = leg_mass(ch, leg1, s);
                mt2 = leg_mass(ch, leg2, s);
            } else if (sideof[i] == 0) {
                leg1 = root->child[order[i]];
                mt1 = leg_mass(ch, leg1, s);
                mt2 = sqrt(sts[i]);
            } else {
                leg1 = root->child[order[i]];
                mt1 = sqrt(sts[i]);
                mt2 = leg_mass(ch, leg1, s);
            }
            double tlo, thi, tabs, jt;
            orc_t_min_max(scur, mA2, mB2, mt1, mt2, &tlo, &thi);
            if (tlo < 0.0) tlo = 0.0;
            if (thi < tlo) { fail = 1; thi = tlo; }
            if (ORC_BOOKKEEPING) {   /* condition number of the |t| range width: both bounds carry rounding relative to |t|_max,
                 * and the Jacobian of the |t| map is proportional to |t|_max - |t|_min; spacelike
                 * incoming legs of a light block make the range a sliver of a large |t| */
                double k = thi > tlo ? thi / (thi - tlo) : 1e300;
                if (k > cond) cond = k;
            }
            fail |= orc_map_nu(r[L.d_tt[i]], 0.0, ch->t_nu, tlo, thi, ch->a, &tabs, &jt);
            double q1[4], q2[4];
            double j22 = orc_two_to_two(r[L.d_tphi[i]], pA, pB, tabs, mt1, mt2, scur, mA2, mB2, q1, q2);
            if (ORC_BOOKKEEPING) {   /* the legs' components and the sampled block invariant agree only to eps E0^2, which the
                 * boost into and out of the block rest frame amplifies by gamma^2 = E0^2/s */
                double e0 = pA[0] + pB[0];
                double g2 = e0 * e0 / scur;
                if (g2 > condp) condp = g2;
            }
            if (ORC_BOOKKEEPING) {
                double gap = scur - (mt1 + mt2) * (mt1 + mt2);
                double k = gap > 0.0 ? scur / gap : 1e300;
                if (k > cond) cond = k;
                if (k > condp) condp = k;
                /* 1 + cos(theta) = (|t|_max - |t|)/B: |t| has ulp error relative to |t|_max; the
                 * backward leg's p_T and the next blocks' frames inherit it */
                double kt = (thi - tabs) > 0.0 ? thi / (thi - tabs) : 1e300;
                if (kt > condp) condp = kt;
            }
            jac *= jt * j22;
            {   /* t-propagator of the SDE product, from the sampled invariant */
                double dd = -tabs - ch->Mt * ch->Mt;
                own_t_props *= 1.0 / (dd * dd);
            }
            if (i == kappa) {
                memcpy(p[leg1], q1, sizeof q1);
                memcpy(p[leg2], q2, sizeof q2);
            } else if (sideof[i] == 0) {
                memcpy(p[leg1], q1, sizeof q1);
                for (int mu = 0; mu < 4; ++mu) pA[mu] -= q1[mu];
                mA2 = -tabs;
                scur = sts[i];
            } else {
                memcpy(p[leg1], q2, sizeof q2);
                for (int mu = 0; mu < 4; ++mu) pB[mu] -= q2[mu];
                mB2 = -tabs;
                scur = sts[i];
            }
        }
    }

    /* decays in pre-order (Sec. 2.2.3); the root decay happens at rest */
    for (int i = 0; i < L.n_pre; ++i) {
        int j = L.preorder[i];
        const orc_node* nd = &ch->node[j];
        int c1 = nd->child[0], c2 = nd->child[1];
        double m1 = leg_mass(ch, c1, s), m2 = leg_mass(ch, c2, s);
        double jd = orc_two_body_decay(r[L.d_dphi[j]], r[L.d_dth[j]], s[j], m1, m2,
                                       j == 0 ? NULL : p[j], p[c1], p[c2]);
        jac *= jd;
        if (ORC_BOOKKEEPING && j != 0) {   /* the parent momentum's rounding, boosted with gamma = E0/m0 */
            double g2 = p[j][0] * p[j][0] / s[j];
            if (g2 > condp) condp = g2;
        }
        if (ORC_BOOKKEEPING) {   /* closeness to threshold: lambda's factor s0 - (m1+m2)^2 amplifies rounding by s0/(...) */
            double gap = s[j] - (m1 + m2) * (m1 + m2);
            double k = gap > 0.0 ? s[j] / gap : 1e300;
            if (k > cond) cond = k;
            if (k > condp) condp = k;
        }
    }

    /* stack [p_a, p_b, p_1..p_n] and boost to the lab (boost_beam) */
    memcpy(mom, pa, sizeof pa);
    memcpy(mom + 4, pb, sizeof pb);
    for (int j = 0; j < ch->n_nodes; ++j)
        if (ch->node[j].kind == 0) memcpy(mom + 4 * (2 + ch->node[j].leaf), p[j], sizeof(double) * 4);
    if (ch->hadronic && !ch->partonic)
        for (int i = 0; i < n + 2; ++i) boost_beam(mom + 4 * i, x1, x2);
    x[0] = x1;
    x[1] = x2;

    /* integrand and multichannel weight */
    double f = 1.0, alpha = 1.0, p_mom = 0.0;
    if (ORC_BOOKKEEPING && ch->hadronic && (ch->integrand == 2 || ch->integrand == 3 || ch->integrand == 4)) {
        /* (1-x)^beta of the parton density: an ulp of x is amplified by beta x/(1-x) */
        double k = fabs(ch->pdf_b) * fmax(x1 / (1.0 - x1), x2 / (1.0 - x2));
        if (k > cond) cond = k;
    }
    if (ch->integrand == 1) {
        const double* q = mom + 8;
        double c = q[3] / sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        f = 1.0 + c * c;
    } else if (ch->integrand == 2) {
        f = (ch->hadronic ? pdf(ch, x1) * pdf(ch, x2) : 1.0) * P_own;
    } else if (ch->integrand == 3 || ch->integrand == 4) {
        /* f = f(x1) f(x2) sum_j P_j; SDE weight alpha_c = P_c / sum_j P_j (integrand 3), or the
         * constant 1/n_channels (integrand 4, used to check that sum_c I_c does not depend on alpha).
         * The channel's own P_c uses its sampled invariants; the others are evaluated from momenta. */
        double Pc = P_own * own_t_props;
        double sum = Pc;
        for (int j = 0; j < sde->n_ch; ++j) if (j != chan) sum += sde_from_momenta(sde, j, mom);
        f = (ch->hadronic ? pdf(ch, x1) * pdf(ch, x2) : 1.0) * sum;
        alpha = (ch->integrand == 3) ? Pc / sum : 1.0 / (double)sde->n_ch;
        p_mom = sde_from_momenta(sde, chan, mom);
    }
    double w = jac * f * alpha;

    /* cut_unphysical (reading: non-finite weight or momenta, or x1, x2 outside (0,1]) */
    int cut = 0;
    if (!isfinite(w)) cut = 1;
    for (int i = 0; i < 4 * (n + 2); ++i) if (!isfinite(mom[i])) cut = 1;
    if (!(x1 > 0.0 && x1 <= 1.0 && x2 > 0.0 && x2 <= 1.0)) cut = 1;
    if (cut) w = 0.0;

    if (alpha_out) *alpha_out = alpha;
    if (aux) {
        aux[AUX_SHAT] = shat; aux[AUX_WPS] = jac; aux[AUX_F] = f; aux[AUX_JV] = jv;
        aux[AUX_POWN] = P_own * own_t_props; aux[AUX_CUT] = cut; aux[AUX_FAIL] = fail; aux[AUX_SPARE] = p_mom;
        aux[AUX_COND] = cond;
        aux[AUX_CONDP] = condp;
    }
    return w;
}

/* Batch driver: r [B][d] row-major; mom [B][n+2][4]; x [B][2]; w, alpha [B]; aux [B][8] (may be NULL). */
void orc_forward_batch(const orc_channel* ch, const orc_sde* sde, int chan, const double* grid, int64_t B,
                       const double* r, double* mom, double* x, double* w, double* alpha, double* aux, int threads)
{
    int d = orc_channel_dims(ch);
    int nm = (ch->n + 2) * 4;
#pragma omp parallel for schedule(static) num_threads(threads)
    for (int64_t e = 0; e < B; ++e)
        w[e] = forward_event(ch, sde, chan, grid, r + e * d, mom + e * nm, x + 2 * e,
                             alpha ? alpha + e : NULL, aux ? aux + e * ORC_NAUX : NULL);
}

/* Philox-driven batch: the random point of event ev0+e is drawn in place. */
void orc_generate_batch(const orc_channel* ch, const orc_sde* sde, int chan, const double* grid,
                        uint64_t seed, uint64_t ev0, int64_t B, double* mom, double* x, double* w,
                        double* alpha, int threads)
{
    int d = orc_channel_dims(ch);
    int nm = (ch->n + 2) * 4;
#pragma omp parallel for schedule(static) num_threads(threads)
    for (int64_t e = 0; e < B; ++e) {
        double r[64], mloc[(ORC_MAXN + 2) * 4], xloc[2], aloc;
        orc_random_point(seed, (uint32_t)chan, ev0 + (uint64_t)e, d, r);
        w[e] = forward_event(ch, sde, chan, grid, r, mloc, xloc, &aloc, NULL);
        if (mom) memcpy(mom + e * nm, mloc, sizeof(double) * nm);
        if (x) { x[2 * e] = xloc[0]; x[2 * e + 1] = xloc[1]; }
        if (alpha) alpha[e] = aloc;
    }
}

/* Per-channel statistics in event order: count, nonzero count, sum w, sum w^2, max w. */
void orc_stats(const double* w, int64_t B, double* out)
{
    double n_nz = 0.0, s1 = 0.0, s2 = 0.0, mx = 0.0;
    for (int64_t e = 0; e < B; ++e) {
        double v = w[e];
        if (v != 0.0) n_nz += 1.0;
        s1 += v;
        s2 += v * v;
        if (v > mx) mx = v;
    }
    out[0] = (double)B; out[1] = n_nz; out[2] = s1; out[3] = s2; out[4] = mx;
}

/* ------------------------------------------------------------------------ */
/* Inverse map (Sec. 2.1: every mapping is invertible; round trip of Sec. 4.1) */
/* ------------------------------------------------------------------------ */
static double unit_phi(double y, double x)
{
    double ph = atan2(y, x) / (2.0 * ORC_PI);
    if (ph < 0.0) ph += 1.0;
    return ph;
}

static void leaf_sum(const orc_channel* ch, int j, const double* mom, double* q)
{
    const orc_node* nd = &ch->node[j];
    if (nd->kind == 0) { for (int mu = 0; mu < 4; ++mu) q[mu] += mom[4 * (2 + nd->leaf) + mu]; return; }
    for (int k = 0; k < nd->nchild; ++k) leaf_sum(ch, nd->child[k], mom, q);
}

static int leaf_list(const orc_channel* ch, int j, int* out, int n)
{
    const orc_node* nd = &ch->node[j];
    if (nd->kind == 0) { out[n] = j; return n + 1; }
    for (int k = 0; k < nd->nchild; ++k) n = leaf_list(ch, nd->child[k], out, n);
    return n;
}

/* (sum_i p_i)^2 = sum_i m_i^2 + sum_{i<j} 2 p_i.p_j with every pair term in the form
 * 2 p_i.p_j = 2 (m_i^2 |p_j|^2 + m_j^2 |p_i|^2 + m_i^2 m_j^2)/(E_i E_j + |p_i||p_j|)
 *             + |p_i||p_j| |n_i - n_j|^2,
 * which keeps full relative precision for nearly collinear pairs. */
static double node_mass2(const orc_channel* ch, int j, const double* mom)
{
    int lv[ORC_MAXN];
    int nl = leaf_list(ch, j, lv, 0);
    double s = 0.0;
    for (int i = 0; i < nl; ++i) s += ch->node[lv[i]].mass * ch->node[lv[i]].mass;
    for (int i = 0; i < nl; ++i)
        for (int k = i + 1; k < nl; ++k) {
            const double* p = mom + 4 * (2 + ch->node[lv[i]].leaf);
            const double* q = mom + 4 * (2 + ch->node[lv[k]].leaf);
            double mp = ch->node[lv[i]].mass, mq = ch->node[lv[k]].mass;
            double ap = sqrt(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
            double aq = sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
            double dx = p[1] / ap - q[1] / aq, dy = p[2] / ap - q[2] / aq, dz = p[3] / ap - q[3] / aq;
            double mterm = 2.0 * (mp * mp * aq * aq + mq * mq * ap * ap + mp * mp * mq * mq) / (p[0] * q[0] + ap * aq);
            s += mterm + ap * aq * (dx * dx + dy * dy + dz * dz);
        }
    return s;
}

/* Recover r from lab momenta [p_a, p_b, p_1..p_n] and (x1, x2). */
static void inverse_event(const orc_channel* ch, const double* grid, const double* mom_lab, const double* xin,
                          double* r)
{
    layout L;
    make_layout(ch, &L);
    const int n = ch->n;
    double mom[(ORC_MAXN + 2) * 4];
    memcpy(mom, mom_lab, sizeof(double) * 4 * (n + 2));
    double x1 = xin[0], x2 = xin[1];
    if (ch->hadronic && !ch->partonic) for (int i = 0; i < n + 2; ++i) unboost_beam(mom + 4 * i, x1, x2);

    double s[ORC_MAXN], p[ORC_MAXN][4];
    int sampled[ORC_MAXN];
    memset(sampled, 0, sizeof sampled);
    for (int j = 0; j < ch->n_nodes; ++j) {
        double q[4] = { 0, 0, 0, 0 };
        leaf_sum(ch, j, mom, q);
        memcpy(p[j], q, sizeof q);
        s[j] = node_mass2(ch, j, mom);
    }
    double shat;
    if (ch->hadronic) {
        shat = x1 * x2 * ch->S;
        double smin = 0.0;
        for (int j = 0; j < ch->n_nodes; ++j) if (ch->node[j].kind == 0) smin += ch->node[j].mass;
        smin *= smin;
        r[L.d_shat] = (ch->shat_G > 0.0) ? orc_inv_bw(shat, ch->shat_M, ch->shat_G, smin, ch->S)
                                         : orc_inv_nu(shat, ch->shat_M, ch->shat_nu, smin, ch->S, ch->a);
        r[L.d_x] = log(x1) / log(shat / ch->S);
    } else shat = ch->sqrt_s * ch->sqrt_s;
    s[0] = shat;
    sampled[0] = 1;
    for (int i = 0; i < ch->n_sorder; ++i) {
        int j = ch->sorder[i];
        const orc_node* nd = &ch->node[j];
        double mlo = min_mass(ch, j, sampled, s);
        double mhi = max_mass(ch, &L, j, sampled, s, NULL);
        double smin = mlo * mlo, smax = mhi * mhi;
        r[L.d_s[j]] = (nd->G > 0.0) ? orc_inv_bw(s[j], nd->M, nd->G, smin, smax)
                                    : orc_inv_nu(s[j], nd->M, nd->nu, smin, smax, ch->a);
        sampled[j] = 1;
    }
    const orc_node* root = &ch->node[0];
    int kappa = (root->kind == 2) ? root->nchild - 1 : 0;
    if (kappa > 0) {
        int order[ORC_MAXK + 1], sideof[ORC_MAXK + 1];
        int left = 0, right = kappa;
        for (int i = 1; i < kappa; ++i) {
            if (ch->tside[i] == 0) { order[i] = left++; sideof[i] = 0; }
            else { order[i] = right--; sideof[i] = 1; }
        }
        order[kappa] = left;
        order[kappa + 1] = right;
        /* remaining-cluster invariants */
        double sts[ORC_MAXK + 1];
        sts[0] = shat;
        int l2 = 0, r2 = kappa;
        for (int i = 1; i < kappa; ++i) {
            if (sideof[i] == 0) ++l2; else --r2;
            double q[4] = { 0, 0, 0, 0 };
            for (int k = l2; k <= r2; ++k) for (int mu = 0; mu < 4; ++mu) q[mu] += p[root->child[k]][mu];
            sts[i] = mdot(q, q);
            double msum = 0.0;
            for (int k = l2; k <= r2; ++k) msum += leg_mass(ch, root->child[k], s);
            double mi = leg_mass(ch, root->child[order[i]], s);
            double mx = sqrt(sts[i - 1]) - mi;
            r[L.d_ts[i]] = orc_inv_nu(sts[i], 0.0, ch->ts_nu, msum * msum, mx * mx, ch->a);
        }
        double pa[4] = { sqrt(shat) / 2, 0, 0, sqrt(shat) / 2 }, pb[4] = { sqrt(shat) / 2, 0, 0, -sqrt(shat) / 2 };
        double pA[4], pB[4];
        memcpy(pA, pa, sizeof pA);
        memcpy(pB, pb, sizeof pB);
        double mA2 = 0.0, mB2 = 0.0, scur = shat;
        for (int i = 1; i <= kappa; ++i) {
            double mt1, mt2, q1[4], q2[4];
            if (i == kappa) {
                int l1 = root->child[order[kappa]], l2b = root->child[order[kappa + 1]];
                mt1 = leg_mass(ch, l1, s); mt2 = leg_mass(ch, l2b, s);
                memcpy(q1, p[l1], sizeof q1); memcpy(q2, p[l2b], sizeof q2);
            } else if (sideof[i] == 0) {
                int l1 = root->child[order[i]];
                mt1 = leg_mass(ch, l1, s); mt2 = sqrt(sts[i]);
                memcpy(q1, p[l1], sizeof q1);
                for (int mu = 0; mu < 4; ++mu) q2[mu] = pA[mu] + pB[mu] - q1[mu];
            } else {
                int l1 = root->child[order[i]];
                mt1 = sqrt(sts[i]); mt2 = leg_mass(ch, l1, s);
                memcpy(q2, p[l1], sizeof q2);
                for (int mu = 0; mu < 4; ++mu) q1[mu] = pA[mu] + pB[mu] - q2[mu];
            }
            double dq[4] = { pA[0] - q1[0], pA[1] - q1[1], pA[2] - q1[2], pA[3] - q1[3] };
            double tabs = -mdot(dq, dq);
            double tlo, thi;
            orc_t_min_max(scur, mA2, mB2, mt1, mt2, &tlo, &thi);
            if (tlo < 0.0) tlo = 0.0;
            r[L.d_tt[i]] = orc_inv_nu(tabs, 0.0, ch->t_nu, tlo, thi, ch->a);
            /* azimuth of q1 around the pA axis in the block rest frame */
            double p0[4] = { pA[0] + pB[0], pA[1] + pB[1], pA[2] + pB[2], pA[3] + pB[3] };
            double m0 = sqrt(scur);
            double pAs[4], q1s[4];
            boost_to_rest(pA, p0, m0, pAs);
            boost_to_rest(q1, p0, m0, q1s);
            double cA, sA, cpA, spA;
            direction(pAs + 1, &cA, &sA, &cpA, &spA);
            /* inverse rotation R^T = Ry(-theta) Rz(-phi) */
            double v1 = cpA * q1s[1] + spA * q1s[2];
            double v2 = -spA * q1s[1] + cpA * q1s[2];
            double v3 = q1s[3];
            double xr = cA * v1 - sA * v3;
            double yr = v2;
            r[L.d_tphi[i]] = unit_phi(yr, xr);
            if (i < kappa) {
                if (sideof[i] == 0) { for (int mu = 0; mu < 4; ++mu) pA[mu] -= q1[mu]; mA2 = -tabs; }
                else { for (int mu = 0; mu < 4; ++mu) pB[mu] -= q2[mu]; mB2 = -tabs; }
                scur = sts[i];
            }
        }
    }
    for (int i = 0; i < L.n_pre; ++i) {
        int j = L.preorder[i];
        const orc_node* nd = &ch->node[j];
        int c1 = nd->child[0];
        double q[4];
        if (j == 0) memcpy(q, p[c1], sizeof q);
        else boost_to_rest(p[c1], p[j], sqrt(s[j]), q);
        double pt2 = q[1] * q[1] + q[2] * q[2];
        double pabs = sqrt(pt2 + q[3] * q[3]);
        /* r_theta = (1 + cos theta)/2, taken as sin^2(theta/2) form near the poles */
        double rth;
        if (q[3] >= 0.0) rth = 1.0 - (pt2 / (pabs * (pabs + q[3]))) / 2.0;
        else rth = (pt2 / (pabs * (pabs - q[3]))) / 2.0;
        r[L.d_dth[j]] = rth;
        r[L.d_dphi[j]] = unit_phi(q[2], q[1]);
    }
    for (int j = 0; j < ch->vegas_dims; ++j)
        r[j] = orc_vegas_inv(r[j], grid + j * (ch->vegas_bins + 1), ch->vegas_bins);
}

void orc_inverse_batch(const orc_channel* ch, const double* grid, int64_t B, const double* mom, const double* x,
                       double* r, int threads)
{
    int d = orc_channel_dims(ch);
    int nm = (ch->n + 2) * 4;
#pragma omp parallel for schedule(static) num_threads(threads)
    for (int64_t e = 0; e < B; ++e) inverse_event(ch, grid, mom + e * nm, x + 2 * e, r + e * d);
}

/* The SDE weight P_j of channel j (products of propagator denominators) for a batch of lab
 * momenta [B][n+2][4]: the channel density numerator of the global multichannel integrand. */
void orc_sde_weights(const orc_sde* sde, int j, int64_t B, int n, const double* mom, double* out)
{
    for (int64_t e = 0; e < B; ++e) out[e] = sde_from_momenta(sde, j, mom + e * (n + 2) * 4);
}

int orc_sizeof_channel(void) { return (int)sizeof(orc_channel); }
int orc_sizeof_sde(void) { return (int)sizeof(orc_sde); }
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#ifdef __cplusplus
}
#endif
