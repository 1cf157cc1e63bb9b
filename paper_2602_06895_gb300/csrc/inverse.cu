// inverse.cu -- the inverse channel map on the GPU (every mapping of Sec. 2 is invertible; the
// round trip of Sec. 4.1) and the global multichannel weight of Kleiss and Pittau (Eq.
// multi-channel-standard).
//
// ps_inverse_kernel recovers, for one event per thread and in FP64, the random numbers r of a
// channel from the lab-frame momenta [p_a, p_b, p_1..p_n] and (x1, x2):
//   - the longitudinal beam boost is undone on the light cone;
//   - every node's invariant comes from its leaves in the collinear-safe chord form
//       (sum p_i)^2 = sum m_i^2 + sum_{i<k} [2 (m_i^2 |p_k|^2 + m_k^2 |p_i|^2 + m_i^2 m_k^2)
//                      / (E_i E_k + |p_i||p_k|) + |p_i||p_k| |n_i - n_k|^2];
//   - shat, x1 x2, the s-channel invariants (with the forward's recursive bounds), the t-chain
//     invariants, |t| of every 2->2 block and its azimuth about p_A in the block rest frame, and
//     the decay angles in each parent's rest frame are passed through the inverse invariant maps;
//   - the VEGAS grid is inverted last.
// The same kernel evaluates the channel's SDE propagator product P(p) from the lab momenta.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "kin.cuh"
#include "ps_internal.h"

namespace ps {
namespace inv {

using dev::kPi;
using dev::P4;

constexpr int kMaxLeg = kMaxOutMomenta + 2;

// inverse power-law map (anchored as the forward map)
__device__ __forceinline__ double inv_nu(double x, double m, double nu, double xmin, double xmax, double a) {
    const double m2 = (m > 0.0) ? m * m : -a;
    const double lo = xmin - m2, hi = xmax - m2;
    const double L = log1p((xmax - xmin) / lo);
    if (nu == 1.0) return log1p((x - xmin) / lo) / L;
    const double w = 1.0 - nu;
    if (nu < 1.0) return expm1(w * log1p((x - xmin) / lo)) / expm1(w * L);
    return 1.0 - expm1(w * log((x - m2) / hi)) / expm1(-w * L);
}

// inverse Breit-Wigner map: the angle measured from the nearer end of the range
__device__ __forceinline__ double inv_bw(double x, double M, double G, double xmin, double xmax) {
    const double mg = M * G, m2 = M * M;
    const double a = (xmin - m2) / mg, b = (xmax - m2) / mg;
    const double D = atan2((xmax - xmin) / mg, fma(a, b, 1.0));
    const double t = (x - m2) / mg;
    if (x - xmin <= xmax - x) return atan2((x - xmin) / mg, fma(a, t, 1.0)) / D;
    return 1.0 - atan2((xmax - x) / mg, fma(b, t, 1.0)) / D;
}

__device__ __forceinline__ double inv_invariant(double x, double M, double G, double nu, double xmin, double xmax,
                                                double a) {
    return G > 0.0 ? inv_bw(x, M, G, xmin, xmax) : inv_nu(x, M, nu, xmin, xmax, a);
}

__device__ __forceinline__ double unit_phi(double y, double x) {
    double ph = atan2(y, x) / (2.0 * kPi);
    return ph < 0.0 ? ph + 1.0 : ph;
}

__device__ __forceinline__ double vegas_inv(double rp, const double* e, int N) {
    int lo = 0, hi = N;  // e[lo] <= rp < e[lo + 1]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (e[mid] <= rp) lo = mid;
        else hi = mid;
    }
    return (static_cast<double>(lo) + (rp - e[lo]) / (e[lo + 1] - e[lo])) / static_cast<double>(N);
}

__global__ void __launch_bounds__(128) ps_inverse_kernel(const __grid_constant__ InvPlan P, int64_t batch,
                                                          const double* mom, int64_t ldm, const double* x1in,
                                                          const double* x2in, const double* grid, double* r,
                                                          int64_t ldr, double* Pout) {
    const int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b >= batch) return;
    const int n = P.n;
    P4 q[kMaxLeg];
    for (int i = 0; i < n + 2; ++i)
        q[i] = {mom[(4 * i) * ldm + b], mom[(4 * i + 1) * ldm + b], mom[(4 * i + 2) * ldm + b],
                mom[(4 * i + 3) * ldm + b]};
    const double x1 = P.hadronic ? x1in[b] : 1.0, x2 = P.hadronic ? x2in[b] : 1.0;

    // SDE propagator product from the lab momenta (q_k = p_a - legs for t-channel propagators)
    if (Pout) {
        double prod = 1.0;
        for (int k = 0; k < P.n_prop; ++k) {
            P4 s = P.pkind[k] == 1 ? q[0] : P4{0.0, 0.0, 0.0, 0.0};
            const double sg = P.pkind[k] == 1 ? -1.0 : 1.0;
            for (int i = 0; i < n; ++i)
                if (P.pmask[k] & (1u << i)) s = {s.e + sg * q[2 + i].e, s.x + sg * q[2 + i].x, s.y + sg * q[2 + i].y,
                                                 s.z + sg * q[2 + i].z};
            const double inv = dev::p4_sq(s);
            const double dd = inv - P.pM[k] * P.pM[k];
            prod *= P.pkind[k] == 1 ? 1.0 / (dd * dd) : 1.0 / (dd * dd + P.pM[k] * P.pM[k] * P.pG[k] * P.pG[k]);
        }
        Pout[b] = prod;
    }

    // partonic frame (light-cone form of the inverse longitudinal boost)
    if (P.hadronic && P.lab_frame) {
        const double rho = sqrt(x1 / x2);
        for (int i = 0; i < n + 2; ++i) {
            const double plus = (q[i].e + q[i].z) / rho, minus = rho * (q[i].e - q[i].z);
            q[i].e = 0.5 * (plus + minus);
            q[i].z = 0.5 * (plus - minus);
        }
    }

    // node momenta, and the invariants of the non-root decay nodes (the root's is shat; leaves
    // carry their masses): the leaf directions are needed only if such a node exists
    double ap[kMaxLeg], nx[kMaxLeg], ny[kMaxLeg], nz[kMaxLeg], ml[kMaxLeg];
    bool any_decay = false;
    for (int j = 1; j < P.n_nodes; ++j) any_decay |= P.node[j].kind == PS_NODE_DECAY;
    for (int j = 0; j < P.n_nodes; ++j)
        if (P.node[j].kind == PS_NODE_LEAF) {
            const int i = P.node[j].leaf;
            ml[i] = P.node[j].mass;
            if (any_decay) {
                const P4 p = q[2 + i];
                const double a = sqrt(p.x * p.x + p.y * p.y + p.z * p.z);
                ap[i] = a;
                nx[i] = p.x / a;
                ny[i] = p.y / a;
                nz[i] = p.z / a;
            }
        }
    P4 pn[kInvNodes];
    double s[kInvNodes];
    for (int j = 1; j < P.n_nodes; ++j) {
        const InvNode& nd = P.node[j];
        if (nd.kind == PS_NODE_LEAF) {
            pn[j] = q[2 + nd.leaf];
            s[j] = nd.mass * nd.mass;
            continue;
        }
        const uint32_t mask = nd.mask;
        P4 acc{0.0, 0.0, 0.0, 0.0};
        double s2 = 0.0;
        for (int i = 0; i < n; ++i) {
            if (!(mask & (1u << i))) continue;
            acc = dev::p4_add(acc, q[2 + i]);
            s2 += ml[i] * ml[i];
            for (int k = i + 1; k < n; ++k) {
                if (!(mask & (1u << k))) continue;
                const double dx = nx[i] - nx[k], dy = ny[i] - ny[k], dz = nz[i] - nz[k];
                const double mi2 = ml[i] * ml[i], mk2 = ml[k] * ml[k];
                s2 += 2.0 * (mi2 * ap[k] * ap[k] + mk2 * ap[i] * ap[i] + mi2 * mk2) /
                          (q[2 + i].e * q[2 + k].e + ap[i] * ap[k]) +
                      ap[i] * ap[k] * (dx * dx + dy * dy + dz * dz);
            }
        }
        pn[j] = acc;
        s[j] = s2;
    }
    auto leg_mass = [&](int j) { return P.node[j].kind == PS_NODE_LEAF ? P.node[j].mass : sqrt(s[j]); };

    double shat;
    if (P.hadronic) {
        shat = x1 * x2 * P.S;
        r[P.d_shat * ldr + b] = inv_invariant(shat, P.shat_M, P.shat_G, P.shat_nu, P.mleaf * P.mleaf, P.S, P.a);
        r[P.d_x * ldr + b] = log(x1) / log(shat / P.S);
    } else {
        shat = P.sqrt_s * P.sqrt_s;
    }
    s[0] = shat;

    // s-channel invariants with the forward's bounds
    for (int i = 0; i < P.n_sorder; ++i) {
        const int j = P.sorder[i];
        double mlo = P.lo_c[i];
        for (int k = P.lo_beg[i]; k < P.off_beg[i]; ++k) mlo += sqrt(s[P.ids[k]]);
        double off = P.off_c[i];
        for (int k = P.off_beg[i]; k < P.lo_beg[i + 1]; ++k) off += sqrt(s[P.ids[k]]);
        const int top = P.top[i];
        const double mtop = (top == 0 && !P.hadronic) ? P.sqrt_s : sqrt(s[top]);
        const double mhi = fmax(mtop - off, mlo);
        const InvNode& nd = P.node[j];
        r[P.d_s[j] * ldr + b] = inv_invariant(s[j], nd.M, nd.G, nd.nu, mlo * mlo, mhi * mhi, P.a);
    }

    // t-chain (legs taken inwards from side A or B)
    const int kappa = P.kappa;
    if (kappa > 0) {
        const InvNode& root = P.node[0];
        double sts[kInvLegs + 1];
        sts[0] = shat;
        int l2 = 0, r2 = kappa;
        for (int i = 1; i < kappa; ++i) {
            if (P.side[i] == 0) ++l2;
            else --r2;
            P4 c{0.0, 0.0, 0.0, 0.0};
            double msum = 0.0;
            for (int k = l2; k <= r2; ++k) {
                c = dev::p4_add(c, pn[root.child[k]]);
                msum += leg_mass(root.child[k]);
            }
            sts[i] = dev::p4_sq(c);
            const double mi = leg_mass(root.child[P.order[i]]);
            const double mx = fmax(sqrt(sts[i - 1]) - mi, 0.0);
            const double smin = msum * msum;
            r[P.d_ts[i] * ldr + b] = inv_nu(sts[i], 0.0, P.ts_nu, smin, fmax(mx * mx, smin), P.a);
        }
        const double e0 = 0.5 * sqrt(shat);
        P4 pA{e0, 0.0, 0.0, e0}, pB{e0, 0.0, 0.0, -e0};
        double mA2 = 0.0, mB2 = 0.0, scur = shat;
        for (int i = 1; i <= kappa; ++i) {
            double m1, m2;
            P4 q1, q2;
            if (i == kappa) {
                const int la = root.child[P.order[kappa]], lb = root.child[P.order[kappa + 1]];
                m1 = leg_mass(la);
                m2 = leg_mass(lb);
                q1 = pn[la];
                q2 = pn[lb];
            } else if (P.side[i] == 0) {
                const int l1 = root.child[P.order[i]];
                m1 = leg_mass(l1);
                m2 = sqrt(sts[i]);
                q1 = pn[l1];
                q2 = dev::p4_sub(dev::p4_add(pA, pB), q1);
            } else {
                const int l1 = root.child[P.order[i]];
                m1 = sqrt(sts[i]);
                m2 = leg_mass(l1);
                q2 = pn[l1];
                q1 = dev::p4_sub(dev::p4_add(pA, pB), q2);
            }
            const double tabs = -dev::p4_sq(dev::p4_sub(pA, q1));
            double tmin, tmax, Bt;
            dev::t_range(scur, mA2, mB2, m1, m2, tmin, tmax, Bt);
            const double tlo = fmax(tmin, 0.0), thi = fmax(tmax, tlo);
            r[P.d_tt[i] * ldr + b] = inv_nu(tabs, 0.0, P.t_nu, tlo, thi, P.a);
            // azimuth of q1 about the direction of pA in the block rest frame
            const P4 p0 = dev::p4_add(pA, pB);
            const double m0 = sqrt(scur);
            const P4 pAs = dev::boost_in(pA, p0, m0), q1s = dev::boost_in(q1, p0, m0);
            const double pt = sqrt(pAs.x * pAs.x + pAs.y * pAs.y);
            const double pp = sqrt(pt * pt + pAs.z * pAs.z);
            const double cA = pAs.z / pp, sA = pt / pp;
            const double cpA = pt > 0.0 ? pAs.x / pt : 1.0, spA = pt > 0.0 ? pAs.y / pt : 0.0;
            const double v1 = cpA * q1s.x + spA * q1s.y;
            const double v2 = -spA * q1s.x + cpA * q1s.y;
            r[P.d_tphi[i] * ldr + b] = unit_phi(v2, cA * v1 - sA * q1s.z);
            if (i < kappa) {
                if (P.side[i] == 0) {
                    pA = dev::p4_sub(pA, q1);
                    mA2 = -tabs;
                } else {
                    pB = dev::p4_sub(pB, q2);
                    mB2 = -tabs;
                }
                scur = sts[i];
            }
        }
    }

    // decay angles in each parent's rest frame (the root decays at rest)
    for (int i = 0; i < P.n_pre; ++i) {
        const int j = P.pre[i];
        const int c1 = P.node[j].child[0];
        const P4 qq = j == 0 ? pn[c1] : dev::boost_in(pn[c1], pn[j], sqrt(s[j]));
        const double pt2 = qq.x * qq.x + qq.y * qq.y;
        const double pa = sqrt(pt2 + qq.z * qq.z);
        // r_theta = (1 + cos theta)/2 in the sin^2(theta/2) form near the poles
        const double rth = qq.z >= 0.0 ? 1.0 - 0.5 * (pt2 / (pa * (pa + qq.z))) : 0.5 * (pt2 / (pa * (pa - qq.z)));
        r[P.d_dth[j] * ldr + b] = rth;
        r[P.d_dphi[j] * ldr + b] = unit_phi(qq.y, qq.x);
    }

    for (int j = 0; j < P.vdims; ++j) r[j * ldr + b] = vegas_inv(r[j * ldr + b], grid + j * (P.vbins + 1), P.vbins);
}

struct GlobalArgs {
    int32_t n_ch;
    double alpha[kMaxChannels];
};

// w = f / sum_j alpha_j g_j with g_j = 1 / J_j (J_j = 0: outside channel j, no density); f is
// the given integrand, or pdf(x1) pdf(x2) sum_j P_j (the SDE propagator sum) when f is null.
__global__ void ps_global_weight_kernel(const __grid_constant__ GlobalArgs A, int64_t batch, const double* J,
                                        int64_t ldj, const double* Pp, int64_t ldp, const double* x1,
                                        const double* x2, double pa, double pb, const double* f, double* w) {
    const int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (b >= batch) return;
    double g = 0.0;
    for (int j = 0; j < A.n_ch; ++j) {
        const double Jj = J[j * ldj + b];
        if (Jj > 0.0) g += A.alpha[j] / Jj;
    }
    double fv;
    if (f) {
        fv = f[b];
    } else {
        double ps = 0.0;
        for (int j = 0; j < A.n_ch; ++j) ps += Pp[j * ldp + b];
        fv = ps;
        if (x1) fv *= pow(x1[b], pa) * pow(1.0 - x1[b], pb) * pow(x2[b], pa) * pow(1.0 - x2[b], pb);
    }
    w[b] = g > 0.0 ? fv / g : 0.0;
}

}  // namespace inv

void count_launches(int n);

int launch_inverse(const InvPlan& plan, int64_t batch, const double* mom, int64_t ld_m, const double* x1,
                   const double* x2, const double* grid, double* r, int64_t ld_r, double* P, void* stream,
                   std::string* err) {
    if (batch <= 0) return PS_OK;
    const unsigned blocks = static_cast<unsigned>((batch + 127) / 128);
    inv::ps_inverse_kernel<<<blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(plan, batch, mom, ld_m, x1, x2,
                                                                                   grid, r, ld_r, P);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("ps_inverse_kernel: ") + cudaGetErrorString(e);
        return PS_ERR_CUDA;
    }
    return PS_OK;
}

int launch_global_weights(int n_ch, int64_t batch, const double* J, int64_t ld_j, const double* P, int64_t ld_p,
                          const double* alpha, const double* x1, const double* x2, double pdf_a, double pdf_b,
                          const double* f, double* w, void* stream, std::string* err) {
    if (batch <= 0) return PS_OK;
    inv::GlobalArgs A{};
    A.n_ch = n_ch;
    for (int j = 0; j < n_ch; ++j) A.alpha[j] = alpha[j];
    const unsigned blocks = static_cast<unsigned>((batch + 255) / 256);
    inv::ps_global_weight_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(A, batch, J, ld_j, P, ld_p, x1,
                                                                                        x2, pdf_a, pdf_b, f, w);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("ps_global_weight_kernel: ") + cudaGetErrorString(e);
        return PS_ERR_CUDA;
    }
    return PS_OK;
}

}  // namespace ps
