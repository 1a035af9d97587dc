// ldpm_adjoint.cu -- reverse (adjoint) pass of the explicit central-difference step.
//
// The paper has no derivatives.  This pass gives the gradient of
//   J = (1/K) sum_{n=1..K} sum_{constrained DOF i} seed_i R_i(t_n)
// (the time mean of seeded reactions R = m a - f) with respect to every facet's E0, alpha and sigma_t,
// by the transpose of the forward recurrences, stepping backward:
//   forward step n:  q_n = q_{n-1} + dt u_{n-1}      (u_{n-1} = v_{n-1/2})
//                    (t_n, h_n) = law(e_n = B q_n, de_n = dt B u_{n-1}, eV_n = C q_n, t_{n-1}, h_{n-1})
//                    f_n = -sum_k D_k^T A_k P_k t_k,   u_n = u_{n-1} + dt M^-1 (f_ext + f_n)  (free DOFs)
//   reverse step n:  a_f = c + dt M^-1 Ubar_n                         (c = -seed / K, constrained DOFs)
//                    a_t = a_t(carried) - A l e(a_f)                  (transposed assembly = the strain
//                                                                        operator on the a_f field)
//                    law VJP -> a_e, a_de, a_eV, a_t(n-1), a_h(n-1), dJ/d(E0, alpha, sigma_t)
//                    Qbar_n = Qbar_{n+1} + B^T a_e + C^T a_eV
//                    Ubar_{n-1} = Ubar_n + dt Qbar_n + dt B^T a_de     (free DOFs; 0 on constrained)
// B^T and C^T have the structure of the forward assembly (facet -> vertex contributions, fixed-order
// sums per tetrahedron vertex, then per particle), so the two launches per reversed step mirror the
// forward pass and are as deterministic.  Non-differentiable points take the derivative of the branch
// the forward value takes; sqrt'(0) is taken as 0.
#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#include "ldpm_device.cuh"
#include "ldpm_internal.h"

namespace ldpm {
namespace {

template <class R>
struct LawVJP {
    V3<R> ae, ade;             // adjoints of the strain and of its increment
    R aeV;                     // adjoint of the tetrahedron's volumetric strain
    R atN, atM, atL, aemax;    // adjoints of the previous history
    R gE0, galpha, gsigma;     // adjoints of the facet's parameters
};

// Reverse of facet_law: given the adjoints (aN, aM, aL, ah) of its outputs (t_N, t_M, t_L, e_max),
// the adjoints of its inputs.  The forward values are recomputed with the expressions of facet_law.
// KT: the tensile reload rule may act (some k_t > 0); without it that code is compiled out.
template <class R, bool KT>
__device__ __forceinline__ void facet_law_vjp(const LawConst<R> &c, R l, V3<R> e, V3<R> de, R eV, R tN, R tM,
                                              R tL, R emax, R aN, R aM, R aL, R ah, LawVJP<R> &o)
{
    const R E0 = c.E0, alpha = c.alpha;
    o.ae = {R(0), R(0), R(0)};
    o.ade = {R(0), R(0), R(0)};
    o.aeV = o.atN = o.atM = o.atL = o.aemax = R(0);
    o.gE0 = o.galpha = o.gsigma = R(0);
    if (c.elastic) {  // t = E0 (e_N, alpha e_M, alpha e_L); e_max unchanged
        const R sT = e.y * aM + e.z * aL;
        o.ae = {E0 * aN, alpha * E0 * aM, alpha * E0 * aL};
        o.gE0 = e.x * aN + alpha * sT;
        o.galpha = E0 * sT;
        o.aemax = ah;
        return;
    }
    if (e.x > R(0)) {
        const R eT2 = e.y * e.y + e.z * e.z;
        const R aT2 = alpha * eT2;
        const R eeff = sqrt(e.x * e.x + aT2);
        if (eeff < c.tiny_strain) {  // elastic limit; e_max = max(e_max, e)
            const R sT = e.y * aM + e.z * aL;
            o.ae = {E0 * aN, alpha * E0 * aM, alpha * E0 * aL};
            o.gE0 = e.x * aN + alpha * sT;
            o.galpha = E0 * sT;
            if (emax > eeff) {
                o.aemax = ah;
            } else if (eeff > R(0)) {
                const R k = ah / eeff;
                o.ae.x += k * e.x;
                o.ae.y += k * alpha * e.y;
                o.ae.z += k * alpha * e.z;
                o.galpha += k * R(0.5) * eT2;
            }
            return;
        }
        // ---- forward values (facet_law, App. A.1)
        const R saT = sqrt(aT2);
        const R omega = atan2(e.x, saT);
        const R inv_e = R(1) / eeff;
        const R sn = e.x * inv_e, cs = saT * inv_e;
        const R sq = sqrt(sn * sn + c.four_alpha_over_r2 * cs * cs);
        const R Dn = sn + sq;
        const R sigma0 = R(2) * c.sigma_t / Dn;
        const R Ht = R(2) * E0 * l / (c.l_t - l);
        const R P = powpos_(omega * R(2.0 / kPi), c.n_t);
        const R H0 = c.Hs_over_alpha + (Ht - c.Hs_over_alpha) * P;
        const R e0 = sigma0 / E0;
        const bool keep = emax > eeff;
        const R emaxp = keep ? emax : eeff;
        const bool soft = emaxp - e0 > R(0);
        const R over = soft ? emaxp - e0 : R(0);
        const R X = exp_(-H0 * over / sigma0);
        const R sigma_bt = sigma0 * X;
        const V3<R> ep = e - de;
        const R epT2 = ep.y * ep.y + ep.z * ep.z;
        const R e_old = sqrt(ep.x * ep.x + alpha * epT2);
        const R num = de.x * (e.x + ep.x) + alpha * (de.y * (e.y + ep.y) + de.z * (e.z + ep.z));
        R d_eff = num / (eeff + e_old);
        const R tT2 = tM * tM + tL * tL;
        const R t_old = sqrt(tN * tN + tT2 * c.inv_alpha);
        bool reload = false;  // k_t > 0: the increment counts only above e_tr
        R e_tr = R(0);
        if (KT && c.k_t > R(0) && t_old <= R(0) && d_eff > R(0)) {
            e_tr = c.k_t * (emaxp - sigma_bt / E0);
            if (e_tr > e_old) {
                reload = true;
                d_eff = eeff > e_tr ? eeff - e_tr : R(0);
            }
        }
        const R tstar = t_old + E0 * d_eff;
        const R t1 = tstar < R(0) ? R(0) : tstar;
        const bool capped = t1 > sigma_bt;
        const R t = capped ? sigma_bt : t1;
        const R r = t * inv_e;
        // ---- reverse.  out = r (e_N, alpha e_M, alpha e_L), r = t / eeff
        const R sT = e.y * aM + e.z * aL;
        const R a_r = e.x * aN + alpha * sT;
        o.ae = {r * aN, alpha * r * aM, alpha * r * aL};
        o.galpha = r * sT;
        const R a_t = a_r * inv_e;
        R a_eeff = -r * inv_e * a_r;
        // vertical return: t = clamp(t*, 0, sigma_bt)
        R a_sbt = R(0), a_tstar = R(0);
        if (capped)
            a_sbt = a_t;
        else if (!(tstar < R(0)))
            a_tstar = a_t;
        // t* = t_old + E0 (eeff - e_old), or t_old + E0 <eeff - e_tr> when reloading past e_tr
        o.gE0 += d_eff * a_tstar;
        const R a_deff = E0 * a_tstar;
        R a_emaxp = ah;
        if (KT && reload) {
            if (eeff > e_tr) {  // e_tr = k_t (e_max - sigma_bt / E0)
                a_eeff += a_deff;
                a_emaxp -= c.k_t * a_deff;
                a_sbt += c.k_t * a_deff / E0;
                o.gE0 -= c.k_t * sigma_bt / (E0 * E0) * a_deff;
            }
        } else {
            a_eeff += a_deff;
            if (e_old > R(0)) {  // e_old = |e - de|_alpha
                const R k = -a_deff / e_old;
                const V3<R> a_ep = {k * ep.x, k * alpha * ep.y, k * alpha * ep.z};
                o.ae = o.ae + a_ep;
                o.ade = o.ade - a_ep;
                o.galpha += k * R(0.5) * epT2;
            }
        }
        if (t_old > R(0)) {  // t_old = sqrt(t_N^2 + (t_M^2 + t_L^2) / alpha)
            const R k = a_tstar / t_old;
            o.atN = k * tN;
            o.atM = k * c.inv_alpha * tM;
            o.atL = k * c.inv_alpha * tL;
            o.galpha -= k * R(0.5) * tT2 * c.inv_alpha * c.inv_alpha;
        }
        // sigma_bt = sigma0 exp(-Y), Y = H0 over / sigma0
        R a_sigma0 = R(0), a_H0 = R(0), a_over = R(0);
        if (a_sbt != R(0)) {
            const R Y = H0 * over / sigma0;
            a_sigma0 = a_sbt * X * (R(1) + Y);
            a_H0 = -a_sbt * X * over;
            a_over = -a_sbt * X * H0;
        }
        // over = <e_max - e0>, e_max = max(e_max_old, eeff)
        R a_e0 = R(0);
        if (soft) {
            a_emaxp += a_over;
            a_e0 = -a_over;
        }
        if (keep)
            o.aemax = a_emaxp;
        else
            a_eeff += a_emaxp;
        // e0 = sigma0 / E0
        a_sigma0 += a_e0 / E0;
        o.gE0 -= e0 / E0 * a_e0;
        // H0 = H_s/alpha + (H_t - H_s/alpha) (2 omega / pi)^n_t, H_t = 2 E0 l / (l_t - l), H_s = r_s E0
        o.gE0 += a_H0 * (P * Ht + (R(1) - P) * c.Hs_over_alpha) / E0;
        o.galpha -= a_H0 * (R(1) - P) * c.Hs_over_alpha / alpha;
        const R a_omega = a_H0 * (Ht - c.Hs_over_alpha) * c.n_t * P / omega;
        // sigma0 = 2 sigma_t / (sn + sqrt(sn^2 + (4 alpha / r^2) cs^2))
        o.gsigma += a_sigma0 * sigma0 / c.sigma_t;
        const R a_Dn = -a_sigma0 * sigma0 / Dn;
        const R a_Q = a_Dn * R(0.5) / sq;
        const R a_sn = a_Dn + a_Q * R(2) * sn;
        const R a_cs = a_Q * R(2) * c.four_alpha_over_r2 * cs;
        o.galpha += a_Q * cs * cs * c.four_over_r2;
        // sn = e_N / eeff, cs = saT / eeff, omega = atan2(e_N, saT)
        o.ae.x += (a_sn + a_omega * cs) * inv_e;
        R a_saT = (a_cs - a_omega * sn) * inv_e;
        a_eeff -= (sn * a_sn + cs * a_cs) * inv_e;
        if (saT > R(0)) {  // saT = sqrt(alpha (e_M^2 + e_L^2))
            const R k = a_saT / saT;
            o.ae.y += k * alpha * e.y;
            o.ae.z += k * alpha * e.z;
            o.galpha += k * R(0.5) * eT2;
        }
        {  // eeff = sqrt(e_N^2 + alpha (e_M^2 + e_L^2))
            const R k = a_eeff * inv_e;
            o.ae.x += k * e.x;
            o.ae.y += k * alpha * e.y;
            o.ae.z += k * alpha * e.z;
            o.galpha += k * R(0.5) * eT2;
        }
        return;
    }
    // ---- compression and friction (App. A.2, A.3): forward values
    const bool unload = !(-tN <= c.sigma_c0);
    const R ENc = unload ? c.Ed : E0;
    const R tn_star = tN + ENc * de.x;
    const R eD = e.x - eV;
    const R eDV = eV + c.beta * eD;
    const bool vneg = eV <= R(0);
    const R absD = fabs(eD);
    const R den = vneg ? eV - c.eV0 : c.eV0;
    const R rDV = vneg ? -absD / den : absD / den;
    const bool macp = rDV - c.kc1 > R(0);
    const R mac = macp ? rDV - c.kc1 : R(0);
    const R den2 = R(1) + c.kc2 * mac;
    const R Hc = (c.Hc0 - c.Hc1) / den2 + c.Hc1;
    const R m_eDV = -eDV;
    int bcase;
    R sigma_bc, o_ = R(0), Yc = R(0), Ex = R(0);
    if (m_eDV <= R(0)) {
        bcase = 1;
        sigma_bc = c.sigma_c0;
    } else if (m_eDV <= c.ec1) {
        bcase = 2;
        o_ = m_eDV - c.ec0 > R(0) ? m_eDV - c.ec0 : R(0);
        sigma_bc = c.sigma_c0 + o_ * Hc;
    } else {
        bcase = 3;
        const R sigma_c1 = c.sigma_c0 + (c.ec1 - c.ec0) * Hc;
        Yc = (m_eDV - c.ec1) * Hc / sigma_c1;
        Ex = exp_(Yc);
        sigma_bc = sigma_c1 * Ex;
    }
    const bool low = tn_star < -sigma_bc;
    const R tn1 = low ? -sigma_bc : tn_star;
    const bool zero = tn1 > R(0);
    const R tn = zero ? R(0) : tn1;
    const R tm_s = tM + alpha * E0 * de.y, tl_s = tL + alpha * E0 * de.z;
    const R ex = exp_(tn * c.inv_sigma_N0);
    const R sigma_bs = c.sigma_s + c.mu_diff_sN0 - c.mu_inf * tn - c.mu_diff_sN0 * ex;
    const R tau2 = tm_s * tm_s + tl_s * tl_s;
    // ---- reverse.  Radial return (t_M, t_L) = sigma_bs u / |u| when |u| > sigma_bs, u the trial.
    R a_tn = aN, aum = aM, aul = aL, a_sbs = R(0);
    if (tau2 > sigma_bs * sigma_bs) {
        const R itau = rsqrt_(tau2);
        const R s = sigma_bs * itau;
        const R au = (aM * tm_s + aL * tl_s) * itau;
        a_sbs = au;
        aum = s * (aM - au * tm_s * itau);
        aul = s * (aL - au * tl_s * itau);
    }
    // sigma_bs(t_N) = sigma_s + mu_d sigma_N0 - mu_inf t_N - mu_d sigma_N0 exp(t_N / sigma_N0)
    a_tn += a_sbs * (-c.mu_inf - c.mu_diff_sN0 * ex * c.inv_sigma_N0);
    o.gsigma += a_sbs * c.r_st;
    // shear trial u = t_old + alpha E0 de
    o.atM = aum;
    o.atL = aul;
    o.ade.y = alpha * E0 * aum;
    o.ade.z = alpha * E0 * aul;
    const R sdd = de.y * aum + de.z * aul;
    o.galpha += E0 * sdd;
    o.gE0 += alpha * sdd;
    // t_N = clamp(t_N*, -sigma_bc, 0), t_N* = t_N,old + E_Nc de_N
    R a_tns = R(0), a_sbc = R(0);
    if (!zero) {
        if (low)
            a_sbc = -a_tn;
        else
            a_tns = a_tn;
    }
    o.atN = a_tns;
    o.ade.x = ENc * a_tns;
    o.gE0 += (unload ? c.Ed_E0 : R(1)) * de.x * a_tns;
    o.aemax = ah;
    if (a_sbc != R(0) && bcase != 1) {
        R a_Hc = R(0), a_eDV = R(0), a_ec0 = R(0), a_ec1 = R(0);
        if (bcase == 2) {  // sigma_c0 + <-eDV - ec0> H_c
            a_Hc = a_sbc * o_;
            if (m_eDV - c.ec0 > R(0)) {
                a_eDV = -a_sbc * Hc;
                a_ec0 = -a_sbc * Hc;
            }
        } else {  // sigma_c1 exp(Z / sigma_c1), Z = (-eDV - ec1) H_c, sigma_c1 = sigma_c0 + (ec1 - ec0) H_c
            const R a_sc1 = a_sbc * Ex * (R(1) - Yc);
            const R a_Z = a_sbc * Ex;
            a_eDV = -a_Z * Hc;
            a_ec1 = -a_Z * Hc + a_sc1 * Hc;
            a_ec0 = -a_sc1 * Hc;
            a_Hc = a_Z * (m_eDV - c.ec1) + a_sc1 * (c.ec1 - c.ec0);
        }
        // H_c = (H_c0 - H_c1) / (1 + kc2 <r_DV - kc1>) + H_c1
        const R a_Hc0 = a_Hc / den2;
        const R a_Hc1 = a_Hc - a_Hc0;
        const R a_rDV = macp ? -a_Hc * (c.Hc0 - c.Hc1) * c.kc2 / (den2 * den2) : R(0);
        R a_eV = R(0), a_eV0 = R(0), a_absD;
        if (vneg) {  // r_DV = -|e_D| / (e_V - e_V0)
            a_absD = -a_rDV / den;
            const R g = a_rDV * absD / (den * den);
            a_eV += g;
            a_eV0 -= g;
        } else {  // r_DV = |e_D| / e_V0
            a_absD = a_rDV / den;
            a_eV0 -= a_rDV * absD / (den * den);
        }
        R a_eD = eD < R(0) ? -a_absD : a_absD;
        a_eV += a_eDV;  // e_DV = e_V + beta e_D
        a_eD += c.beta * a_eDV;
        o.ae.x += a_eD;  // e_D = e_N - e_V
        a_eV -= a_eD;
        o.aeV = a_eV;
        // e_c0 = sigma_c0 / E0, e_c1 = kc0 e_c0, e_V0 = kc3 e_c0, H_c0 = (H_c0/E0) E0, H_c1 = (H_c1/E0) E0
        a_ec0 += c.kc0 * a_ec1 + c.kc3 * a_eV0;
        o.gE0 += -c.ec0 / E0 * a_ec0 + c.Hc0_E0 * a_Hc0 + c.Hc1_E0 * a_Hc1;
    }
}

// Reverse facet pass of one step (8 tetrahedra, 96 threads per block).
//   phase A  4 threads per tetrahedron: the forward vertex records of the step (as the forward facet
//            pass), the a_f record, differences to vertex 0; e_V and grad(e_V) per vertex;
//   phase B  one thread per facet: strain and increment (as forward), a_t = carried - A P^T [[a_f]],
//            the law VJP, the new carry, the parameter gradients, and the facet's contributions to
//            its two vertices: displacement adjoints from a_e and velocity adjoints from a_de;
//   phase C  12 threads per tetrahedron: fixed-order sums per vertex over its 6 facets (as forward),
//            plus grad(e_V) times the tetrahedron's summed e_V adjoint.
constexpr int kATets = 8;
constexpr int kARow = 16;  // state row: dx(3) du(3) dv(3) theta(3) omega(3) pad
constexpr int kAFr = 8;    // a_f row: da_u(3) a_theta(3) pad(2)
constexpr int kACon = 24;  // facet contributions: vertex a: q(6) u(6), vertex b: q(6) u(6)
// The contributions are stored vertex-major, as in the forward warp kernel: plane 2 s + h (s = 0..5
// the facet's position in its vertex's fixed summation order, h = 0 for the q half, 1 for the u half)
// holds 6 values per vertex of the tile, so the vertex sums of task t = 12 j + 3 v + q read words
// 2t, 2t + 1 of each plane (contiguous, no bank conflicts).
constexpr int kAPlane = 6 * 4 * kATets + 2;

// Mixed mode: 8 resident blocks per SM.  The register cap (80 per thread) costs 24 bytes of spills
// and doubles the occupancy of the uncapped build; measured 10 % faster on GB300.  The FP64 build
// (bound by the FP64 pipe) keeps its registers.  S1: one specimen in mixed mode, law constants from
// the kernel parameters (m.law1) instead of the global array, as in the forward facet pass.
template <class R, bool KT, bool S1>
__global__ void __launch_bounds__(12 * kATets, sizeof(R) == 4 ? 8 : 1)
    adjoint_facet_kernel(const __grid_constant__ DeviceModel m, AdjointModel a)
{
    using T4 = R4<R>;
    constexpr int TETS = kATets;
    __shared__ alignas(16) R sv[TETS * 4][kARow + 2];
    __shared__ alignas(16) R sa[TETS * 4][kAFr];
    __shared__ alignas(16) R spl[12 * kAPlane];
    __shared__ R sgrad[TETS][4][3];
    __shared__ R saeV[12 * TETS];
    __shared__ R seV[TETS];
    __shared__ int sok[TETS];
    const T4 *__restrict__ geo = static_cast<const T4 *>(m.geo);
    const T4 *__restrict__ hsrc = static_cast<const T4 *>(a.snap_h);
    T4 *__restrict__ adj_h = static_cast<T4 *>(a.adj_h);
    T4 *__restrict__ gacc = static_cast<T4 *>(a.gacc);
    R *__restrict__ tvc2 = static_cast<R *>(a.tvc2);
    const LawConst<R> *__restrict__ lawc = static_cast<const LawConst<R> *>(m.law);

    const int tid = threadIdx.x;
    const int64_t tet0 = (int64_t)blockIdx.x * TETS;
    const int j = tid / 12;
    const int slot = tid - 12 * j;
    const int64_t f = tet0 * 12 + tid;
    const bool valid = tet0 + j < m.T;
    T4 g{}, h{}, car{}, pp{};
    if (valid) {
        g = geo[f];
        h = hsrc[f];
        car = adj_h[f];
        if (m.pf) pp = static_cast<const T4 *>(m.pf)[f];
    }

    // ---- phase A
    if (tid < 4 * TETS) {
        const int jt = tid >> 2, vi = tid & 3;
        const int64_t tt = tet0 + jt;
        int p = -1;
        if (tt < m.T) p = reinterpret_cast<const int *>(m.tet)[4 * tt + vi];
        const int base = (threadIdx.x & 31) & ~3;
        R o[kARow], af[kAFr];
        if constexpr (sizeof(R) == 4) {
            const float *src = static_cast<const float *>(a.snap_p);
            float rec[24], arec[12];
            if (p >= 0) {
                const float4 *r4 = reinterpret_cast<const float4 *>(src + kMirror * (int64_t)p);
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const float4 w = r4[k];
                    rec[4 * k] = w.x;
                    rec[4 * k + 1] = w.y;
                    rec[4 * k + 2] = w.z;
                    rec[4 * k + 3] = w.w;
                }
                const float4 *a4 = reinterpret_cast<const float4 *>(static_cast<const float *>(a.af) + 12 * (int64_t)p);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float4 w = a4[k];
                    arec[4 * k] = w.x;
                    arec[4 * k + 1] = w.y;
                    arec[4 * k + 2] = w.z;
                    arec[4 * k + 3] = w.w;
                }
            } else {
#pragma unroll
                for (int k = 0; k < 24; ++k) rec[k] = 0.0f;
#pragma unroll
                for (int k = 0; k < 12; ++k) arec[k] = 0.0f;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float x0h = __shfl_sync(0xffffffffu, rec[k], base);
                const float x0l = __shfl_sync(0xffffffffu, rec[3 + k], base);
                const float u0h = __shfl_sync(0xffffffffu, rec[6 + k], base);
                const float u0l = __shfl_sync(0xffffffffu, rec[9 + k], base);
                const float v0 = __shfl_sync(0xffffffffu, rec[15 + k], base);
                const float a0h = __shfl_sync(0xffffffffu, arec[k], base);
                const float a0l = __shfl_sync(0xffffffffu, arec[3 + k], base);
                o[k] = (rec[k] - x0h) + (rec[3 + k] - x0l);
                o[3 + k] = (rec[6 + k] - u0h) + (rec[9 + k] - u0l);
                o[6 + k] = rec[15 + k] - v0;
                o[9 + k] = rec[12 + k];
                o[12 + k] = rec[18 + k];
                af[k] = (arec[k] - a0h) + (arec[3 + k] - a0l);
                af[3 + k] = arec[6 + k];
            }
        } else {
            const double *src = static_cast<const double *>(a.snap_p);
            double rec[16], arec[8];
            if (p >= 0) {
                const double2 *r2 = reinterpret_cast<const double2 *>(src + 16 * (int64_t)p);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const double2 w = r2[k];
                    rec[2 * k] = w.x;
                    rec[2 * k + 1] = w.y;
                }
                const double2 *a2 = reinterpret_cast<const double2 *>(static_cast<const double *>(a.af) + 8 * (int64_t)p);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double2 w = a2[k];
                    arec[2 * k] = w.x;
                    arec[2 * k + 1] = w.y;
                }
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) rec[k] = 0.0;
#pragma unroll
                for (int k = 0; k < 6; ++k) arec[k] = 0.0;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double x0 = __shfl_sync(0xffffffffu, rec[k], base);
                const double u0 = __shfl_sync(0xffffffffu, rec[3 + k], base);
                const double v0 = __shfl_sync(0xffffffffu, rec[9 + k], base);
                const double a0 = __shfl_sync(0xffffffffu, arec[k], base);
                o[k] = rec[k] - x0;
                o[3 + k] = rec[3 + k] - u0;
                o[6 + k] = rec[9 + k] - v0;
                o[9 + k] = rec[6 + k];
                o[12 + k] = rec[12 + k];
                af[k] = arec[k] - a0;
                af[3 + k] = arec[3 + k];
            }
        }
        o[15] = R(0);
        af[6] = af[7] = R(0);
#pragma unroll
        for (int k = 0; k < kARow; ++k) sv[tid][k] = o[k];
#pragma unroll
        for (int k = 0; k < kAFr; ++k) sa[tid][k] = af[k];
        // e_V = (1/3) sum_i du_i . (dx_i1 x dx_i2) / det (vertex 0 carries no difference); its gradient
        // with respect to u_i is (dx_i1 x dx_i2) / (3 det), and minus their sum for vertex 0.
        const V3<R> dxs = {o[0], o[1], o[2]};
        const V3<R> dus = {o[3], o[4], o[5]};
        const int i1 = vi == 3 ? 1 : vi + 1;
        const int i2 = i1 == 3 ? 1 : i1 + 1;
        V3<R> a1, a2;
        a1.x = __shfl_sync(0xffffffffu, dxs.x, base + i1);
        a1.y = __shfl_sync(0xffffffffu, dxs.y, base + i1);
        a1.z = __shfl_sync(0xffffffffu, dxs.z, base + i1);
        a2.x = __shfl_sync(0xffffffffu, dxs.x, base + i2);
        a2.y = __shfl_sync(0xffffffffu, dxs.y, base + i2);
        a2.z = __shfl_sync(0xffffffffu, dxs.z, base + i2);
        V3<R> cr = cross(a1, a2);
        if (vi == 0) cr = {R(0), R(0), R(0)};
        R term = dot(dus, cr);
        R det = vi == 0 ? R(0) : dot(dxs, cr);
        term += __shfl_xor_sync(0xffffffffu, term, 1);
        term += __shfl_xor_sync(0xffffffffu, term, 2);
        det = __shfl_sync(0xffffffffu, det, base + 1);
        const bool okt = __shfl_sync(0xffffffffu, p, base) >= 0 && det != R(0);
        const R s3 = okt ? R(1) / (R(3) * det) : R(0);
        V3<R> gv = s3 * cr;
        V3<R> gsum = gv;
#pragma unroll
        for (int off = 1; off < 4; off <<= 1) {
            gsum.x += __shfl_xor_sync(0xffffffffu, gsum.x, off);
            gsum.y += __shfl_xor_sync(0xffffffffu, gsum.y, off);
            gsum.z += __shfl_xor_sync(0xffffffffu, gsum.z, off);
        }
        if (vi == 0) gv = {-gsum.x, -gsum.y, -gsum.z};
        sgrad[jt][vi][0] = gv.x;
        sgrad[jt][vi][1] = gv.y;
        sgrad[jt][vi][2] = gv.z;
        if (vi == 0) {
            seV[jt] = (p >= 0 && det != R(0)) ? term / (R(3) * det) : R(0);
            sok[jt] = p >= 0;
        }
    }
    __syncthreads();

    // ---- phase B
    const bool live = valid && sok[j];
    R cs[kACon];
#pragma unroll
    for (int k = 0; k < kACon; ++k) cs[k] = R(0);
    R aeV = R(0);
    if (live) {
        const int e = slot >> 1;
        const int va = (0x211000 >> (4 * e)) & 0xF;
        const int vb = (0x332321 >> (4 * e)) & 0xF;
        R A[kARow], B[kARow];
#pragma unroll
        for (int k = 0; k < kARow; ++k) {
            A[k] = sv[4 * j + va][k];
            B[k] = sv[4 * j + vb][k];
        }
        const V3<R> d = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        const R inv_l = rsqrt_(dot(d, d));
        const R l = dot(d, d) * inv_l;
        const V3<R> n = inv_l * d;
        V3<R> mt, lt;
        tangent_frame(n, mt, lt);
        const V3<R> ca = {g.x, g.y, g.z};
        const V3<R> cb = ca - d;
        const LawConst<R> *lbase;
        if constexpr (S1 && sizeof(R) == 4) {
            lbase = reinterpret_cast<const LawConst<R> *>(&m.law1);
        } else {
            const int sp = m.tile_spec ? m.tile_spec[tet0 / 32] : 0;
            lbase = lawc + sp;
        }
        LawConst<R> cpf;
        if (m.pf) cpf = facet_params(*lbase, pp.x, pp.y, pp.z);
        const LawConst<R> &c = m.pf ? cpf : *lbase;
        const V3<R> thA = {A[9], A[10], A[11]}, thB = {B[9], B[10], B[11]};
        const V3<R> du = {B[3] - A[3], B[4] - A[4], B[5] - A[5]};
        const V3<R> jump = du + cross(thB, cb) - cross(thA, ca);
        const V3<R> e3 = {dot(n, jump) * inv_l, dot(mt, jump) * inv_l, dot(lt, jump) * inv_l};
        const V3<R> omA = {A[12], A[13], A[14]}, omB = {B[12], B[13], B[14]};
        const V3<R> dv = {B[6] - A[6], B[7] - A[7], B[8] - A[8]};
        const V3<R> djump = dv + cross(omB, cb) - cross(omA, ca);
        const R sdt = c.dt * inv_l;
        const V3<R> de3 = {dot(n, djump) * sdt, dot(mt, djump) * sdt, dot(lt, djump) * sdt};
        // a_t = carried + d J / d t through f_n: -A P^T [[a_f]]
        const V3<R> fA = {sa[4 * j + va][0], sa[4 * j + va][1], sa[4 * j + va][2]};
        const V3<R> fB = {sa[4 * j + vb][0], sa[4 * j + vb][1], sa[4 * j + vb][2]};
        const V3<R> tA = {sa[4 * j + va][3], sa[4 * j + va][4], sa[4 * j + va][5]};
        const V3<R> tB = {sa[4 * j + vb][3], sa[4 * j + vb][4], sa[4 * j + vb][5]};
        const V3<R> jf = (fB - fA) + cross(tB, cb) - cross(tA, ca);
        const R Ar = g.w;
        const R aN = car.x - Ar * dot(n, jf);
        const R aM = car.y - Ar * dot(mt, jf);
        const R aL = car.z - Ar * dot(lt, jf);
        LawVJP<R> o;
        facet_law_vjp<R, KT>(c, l, e3, de3, seV[j], h.x, h.y, h.z, h.w, aN, aM, aL, car.w, o);
        T4 nc;
        nc.x = o.atN;
        nc.y = o.atM;
        nc.z = o.atL;
        nc.w = o.aemax;
        adj_h[f] = nc;
        T4 ga = gacc[f];
        ga.x += o.gE0;
        ga.y += o.galpha;
        ga.z += o.gsigma;
        gacc[f] = ga;
        aeV = o.aeV;
        // e = P^T [[q]] / l and de = dt P^T [[v]] / l: the adjoints pulled back to the jump are
        // Ge = P a_e / l and Gd = dt P a_de / l; vertex a receives -G and -c_a x G, vertex b +G, c_b x G
        const V3<R> Ge = inv_l * (o.ae.x * n + o.ae.y * mt + o.ae.z * lt);
        const V3<R> Gd = sdt * (o.ade.x * n + o.ade.y * mt + o.ade.z * lt);
        const V3<R> Mae = cross(ca, Ge), Mbe = cross(cb, Ge);
        const V3<R> Mad = cross(ca, Gd), Mbd = cross(cb, Gd);
        cs[0] = -Ge.x;
        cs[1] = -Ge.y;
        cs[2] = -Ge.z;
        cs[3] = -Mae.x;
        cs[4] = -Mae.y;
        cs[5] = -Mae.z;
        cs[6] = -Gd.x;
        cs[7] = -Gd.y;
        cs[8] = -Gd.z;
        cs[9] = -Mad.x;
        cs[10] = -Mad.y;
        cs[11] = -Mad.z;
        cs[12] = Ge.x;
        cs[13] = Ge.y;
        cs[14] = Ge.z;
        cs[15] = Mbe.x;
        cs[16] = Mbe.y;
        cs[17] = Mbe.z;
        cs[18] = Gd.x;
        cs[19] = Gd.y;
        cs[20] = Gd.z;
        cs[21] = Mbd.x;
        cs[22] = Mbd.y;
        cs[23] = Mbd.z;
    }
    {
        // edge e = slot / 2 joins local vertices va < vb; it is the ka-th edge of va and the kb-th of
        // vb (ascending), so this facet is entry 2 ka + slot % 2 of va's order, 2 kb + slot % 2 of vb's
        using V2 = typename VecT<R>::v2;
        const int e = slot >> 1, sw = slot & 1;
        const int va = (0x211000 >> (4 * e)) & 0xF, vb = (0x332321 >> (4 * e)) & 0xF;
        const int ka = (0x221210 >> (4 * e)) & 0xF, kb = (0x211000 >> (4 * e)) & 0xF;
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            R *da = spl + (2 * (2 * ka + sw) + hf) * kAPlane + 6 * (4 * j + va);
            R *db = spl + (2 * (2 * kb + sw) + hf) * kAPlane + 6 * (4 * j + vb);
#pragma unroll
            for (int c = 0; c < 6; c += 2) {
                *reinterpret_cast<V2 *>(da + c) = V2{cs[6 * hf + c], cs[6 * hf + c + 1]};
                *reinterpret_cast<V2 *>(db + c) = V2{cs[12 + 6 * hf + c], cs[12 + 6 * hf + c + 1]};
            }
        }
    }
    saeV[tid] = aeV;
    __syncthreads();

    // ---- phase C: thread `slot` of tetrahedron j: vertex v = slot / 3, components 2 q, 2 q + 1 of
    // both halves (q = slot % 3), over the vertex's 3 edges (ascending), each edge's two facets
    if (live) {
        using V2 = typename VecT<R>::v2;
        const int v = slot / 3;
        const int q = slot - 3 * v;
        R s[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
        for (int sp = 0; sp < 6; ++sp) {
            const V2 xq = *reinterpret_cast<const V2 *>(spl + (2 * sp) * kAPlane + 2 * tid);
            const V2 xu = *reinterpret_cast<const V2 *>(spl + (2 * sp + 1) * kAPlane + 2 * tid);
            s[0] += xq.x;
            s[1] += xq.y;
            s[2] += xu.x;
            s[3] += xu.y;
        }
        if (q < 2) {  // displacement components 0..2 also receive grad(e_V) times the summed a_eV
            R aT = R(0);
#pragma unroll
            for (int k = 0; k < 12; ++k) aT += saeV[12 * j + k];
            if (2 * q < 3) s[0] += aT * sgrad[j][v][2 * q];
            if (2 * q + 1 < 3) s[1] += aT * sgrad[j][v][2 * q + 1];
        }
        R *dst = tvc2 + (tet0 + j) * 48 + 12 * v;
        dst[2 * q] = s[0];
        dst[2 * q + 1] = s[1];
        dst[6 + 2 * q] = s[2];
        dst[6 + 2 * q + 1] = s[3];
    }
}

// Reverse particle pass: 8 lanes per particle sum its (tetrahedron, vertex) slots in CSR order, then
// lanes 0..5 update one DOF each: Qbar += g_q; Ubar += dt Qbar + g_u; a_f = c + dt Ubar / m (free DOFs;
// constrained DOFs keep Qbar = Ubar = 0, a_f = c).
template <class R>
__global__ void __launch_bounds__(256) adjoint_gather_kernel(DeviceModel m, AdjointModel a)
{
    constexpr int LPP = 8;
    const int32_t *__restrict__ ent = static_cast<const int32_t *>(m.ent);
    const R *__restrict__ tvc2 = static_cast<const R *>(a.tvc2);
    const int lane = threadIdx.x & 31;
    const int sub = lane & (LPP - 1);
    const int64_t p = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / LPP) + lane / LPP;
    const bool valid = p < m.N;
    int r0 = 0, r1 = 0;
    if (valid) {
        r0 = m.row[p];
        r1 = m.row[p + 1];
    }
    // a slot is 12 values (48 B mixed, 96 B FP64): 16-byte vector loads, two slots in flight
    using V = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
    constexpr int NV = 12 * (int)sizeof(R) / 16;
    constexpr int PER = 16 / (int)sizeof(R);
    R s[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = R(0);
    for (int r = r0 + sub; r < r1; r += 2 * LPP) {
        int id[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) id[k] = (r + k * LPP < r1) ? ent[r + k * LPP] : -1;
        V w[2][NV];
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (id[k] >= 0) {
                const V *src = reinterpret_cast<const V *>(tvc2 + 12 * (int64_t)id[k]);
#pragma unroll
                for (int q = 0; q < NV; ++q) w[k][q] = src[q];
            }
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (id[k] >= 0) {
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    const R *e = reinterpret_cast<const R *>(&w[k][q]);
#pragma unroll
                    for (int c = 0; c < PER; ++c) s[q * PER + c] += e[c];
                }
            }
    }
#pragma unroll
    for (int off = LPP / 2; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < 12; ++k) s[k] += __shfl_xor_sync(0xffffffffu, s[k], off);
    const bool act = valid && sub < 6;
    const int d = sub < 6 ? sub : 0;
    R gq = s[0], gu = s[6];
#pragma unroll
    for (int k = 1; k < 6; ++k)
        if (d == k) {
            gq = s[k];
            gu = s[6 + k];
        }
    if (!act) return;
    const double *pc = m.pconst + 8 * p;
    const int mask = (int)(((uint64_t)__double_as_longlong(pc[6]) >> (8 * d)) & 0xffu);
    const double dt = m.spec[(int)__double_as_longlong(pc[7])].dt;
    const double cseed = a.cseed[6 * p + d];
    double Q = 0.0, U = 0.0, afv = cseed;
    if (mask == 0) {
        Q = a.Qbar[6 * p + d] + to_double<R>(gq);
        U = a.Ubar[6 * p + d] + dt * Q + to_double<R>(gu);
        afv = cseed + dt * pc[d] * U;
    }
    a.Qbar[6 * p + d] = Q;
    a.Ubar[6 * p + d] = U;
    if constexpr (sizeof(R) == 4) {
        float *rec = static_cast<float *>(a.af) + 12 * p;
        if (d < 3) {
            float hi, lo;
            d2f_split(afv, hi, lo);
            rec[d] = hi;
            rec[3 + d] = lo;
        } else {
            rec[6 + d - 3] = d2f_trunc(afv);
        }
    } else {
        static_cast<double *>(a.af)[8 * p + d] = afv;
    }
}

// a_f = c, Qbar = Ubar = 0 (adj_h, gacc, gsum are cleared with memsets).
template <class R>
__global__ void __launch_bounds__(256) adjoint_init_kernel(DeviceModel m, AdjointModel a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * (int64_t)m.N) return;
    const int64_t p = i / 6;
    const int d = (int)(i - 6 * p);
    const double c = a.cseed[i];
    a.Qbar[i] = 0.0;
    a.Ubar[i] = 0.0;
    if constexpr (sizeof(R) == 4) {
        float *rec = static_cast<float *>(a.af) + 12 * p;
        if (d < 3) {
            float hi, lo;
            d2f_split(c, hi, lo);
            rec[d] = hi;
            rec[3 + d] = lo;
        } else {
            rec[6 + d - 3] = d2f_trunc(c);
        }
        if (d == 0) rec[9] = rec[10] = rec[11] = 0.0f;
    } else {
        double *rec = static_cast<double *>(a.af) + 8 * p;
        rec[d] = c;
        if (d == 0) rec[6] = rec[7] = 0.0;
    }
}

template <class R>
__global__ void __launch_bounds__(256) adjoint_fold_kernel(int64_t nf, AdjointModel a)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    R4<R> *ga = static_cast<R4<R> *>(a.gacc);
    const R4<R> v = ga[f];
    double *gs = a.gsum + 4 * f;
    gs[0] += to_double<R>(v.x);
    gs[1] += to_double<R>(v.y);
    gs[2] += to_double<R>(v.z);
    R4<R> z{};
    ga[f] = z;
}

// One thread per particle: jacc[p] += sum_d (-c_pd) R_pd(t_n) after forward step n, where on a fixed
// DOF R = -f and on a prescribed one R = m vb (ramp(t_n + dt/2) - ramp(t_n - dt/2)) / dt - f.
__global__ void __launch_bounds__(256) objective_kernel(DeviceModel m, AdjointModel a)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m.N) return;
    const double *pc = m.pconst + 8 * p;
    const uint64_t bc = (uint64_t)__double_as_longlong(pc[6]);
    if (bc == 0) return;
    const SpecDyn &S = m.spec[(int)__double_as_longlong(pc[7])];
    const double t = (double)(*m.step) * S.dt;
    const double dr = (ramp(t + S.half_dt, S.inv_ramp) - ramp(t - S.half_dt, S.inv_ramp)) * S.inv_dt;
    double acc = 0.0;
    for (int d = 0; d < 6; ++d) {
        const int mask = (int)((bc >> (8 * d)) & 0xffu);
        if (mask == 0) continue;
        double R_ = -m.pdyn[8 * p + d];
        if (mask == 2) R_ += m.bc_vm[6 * p + d] * dr;
        acc -= a.cseed[6 * p + d] * R_;
    }
    a.jacc[p] += acc;
}

// Test hook: the law and its VJP on independent rows (layouts in ldpm_internal.h).
template <class R>
__global__ void __launch_bounds__(128) law_vjp_kernel(const LawConst<R> *law, int64_t n, const double *in,
                                                      const double *adj_out, double *out, double *adj_in)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *x = in + 16 * i;
    const double *ao = adj_out + 4 * i;
    const LawConst<R> c = facet_params(*law, R(x[12]), R(x[13]), R(x[14]));
    const R l = R(x[0]);
    const V3<R> e = {R(x[1]), R(x[2]), R(x[3])}, de = {R(x[4]), R(x[5]), R(x[6])};
    const R eV = R(x[7]);
    R tN = R(x[8]), tM = R(x[9]), tL = R(x[10]), em = R(x[11]);
    LawVJP<R> o;
    facet_law_vjp<R, true>(c, l, e, de, eV, tN, tM, tL, em, R(ao[0]), R(ao[1]), R(ao[2]), R(ao[3]), o);
    facet_law(c, l, e, de, eV, tN, tM, tL, em);
    double *y = out + 4 * i;
    y[0] = tN;
    y[1] = tM;
    y[2] = tL;
    y[3] = em;
    double *g = adj_in + 16 * i;
    const R v[16] = {R(0), o.ae.x, o.ae.y, o.ae.z, o.ade.x, o.ade.y, o.ade.z, o.aeV,
                     o.atN, o.atM, o.atL, o.aemax, o.gE0, o.galpha, o.gsigma, R(0)};
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] = v[k];
}

}  // namespace

template <class R>
cudaError_t launch_adjoint_init(const DeviceModel &m, const AdjointModel &a, cudaStream_t s)
{
    const int64_t n6 = 6 * (int64_t)m.N, nf = 12 * (int64_t)m.T;
    cudaError_t e = cudaMemsetAsync(a.adj_h, 0, nf * sizeof(R4<R>), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.gacc, 0, nf * sizeof(R4<R>), s);
    if (e == cudaSuccess && a.gsum) e = cudaMemsetAsync(a.gsum, 0, nf * 4 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    if (n6 > 0) adjoint_init_kernel<R><<<(unsigned)((n6 + 255) / 256), 256, 0, s>>>(m, a);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_adjoint_facet(const DeviceModel &m, const AdjointModel &a, cudaStream_t s)
{
    const unsigned fblocks = (unsigned)((m.T + kATets - 1) / kATets);
    if (fblocks) {
        const bool s1 = sizeof(R) == 4 && m.n_spec == 1;
        if (a.reload) {
            if (s1)
                adjoint_facet_kernel<R, true, true><<<fblocks, 12 * kATets, 0, s>>>(m, a);
            else
                adjoint_facet_kernel<R, true, false><<<fblocks, 12 * kATets, 0, s>>>(m, a);
        } else {
            if (s1)
                adjoint_facet_kernel<R, false, true><<<fblocks, 12 * kATets, 0, s>>>(m, a);
            else
                adjoint_facet_kernel<R, false, false><<<fblocks, 12 * kATets, 0, s>>>(m, a);
        }
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_adjoint_gather(const DeviceModel &m, const AdjointModel &a, cudaStream_t s)
{
    const int64_t warps = ((int64_t)m.N + 3) / 4;
    const unsigned gblocks = (unsigned)((warps * 32 + 255) / 256);
    if (gblocks) adjoint_gather_kernel<R><<<gblocks, 256, 0, s>>>(m, a);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_adjoint_fold(const DeviceModel &m, const AdjointModel &a, cudaStream_t s)
{
    const int64_t nf = 12 * (int64_t)m.T;
    if (nf > 0) adjoint_fold_kernel<R><<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(nf, a);
    return cudaGetLastError();
}

cudaError_t launch_objective(const DeviceModel &m, const AdjointModel &a, cudaStream_t s)
{
    if (m.N > 0) objective_kernel<<<(unsigned)((m.N + 255) / 256), 256, 0, s>>>(m, a);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_law_vjp(const LawConst<R> *law, int64_t n, const double *in, const double *adj_out, double *out,
                           double *adj_in, cudaStream_t s)
{
    if (n > 0) law_vjp_kernel<R><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(law, n, in, adj_out, out, adj_in);
    return cudaGetLastError();
}

template cudaError_t launch_adjoint_init<float>(const DeviceModel &, const AdjointModel &, cudaStream_t);
template cudaError_t launch_adjoint_init<double>(const DeviceModel &, const AdjointModel &, cudaStream_t);
template cudaError_t launch_adjoint_facet<float>(const DeviceModel &, const AdjointModel &, cudaStream_t);
template cudaError_t launch_adjoint_facet<double>(const DeviceModel &, const AdjointModel &, cudaStream_t);
template cudaError_t launch_adjoint_gather<float>(const DeviceModel &, const AdjointModel &, cudaStream_t);
template cudaError_t launch_adjoint_gather<double>(const DeviceModel &, const AdjointModel &, cudaStream_t);
template cudaError_t launch_adjoint_fold<float>(const DeviceModel &, const AdjointModel &, cudaStream_t);
template cudaError_t launch_adjoint_fold<double>(const DeviceModel &, const AdjointModel &, cudaStream_t);
template cudaError_t launch_law_vjp<float>(const LawConst<float> *, int64_t, const double *, const double *, double *,
                                           double *, cudaStream_t);
template cudaError_t launch_law_vjp<double>(const LawConst<double> *, int64_t, const double *, const double *,
                                            double *, double *, cudaStream_t);

}  // namespace ldpm
