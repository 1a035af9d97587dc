// ldpm_kernels.cu -- sm_103a kernels of the LDPM explicit central-difference step.
//
// One step (paper Sec. 3, central difference with lumped mass) is two launches.  Between steps the
// state is kept drifted: q_{n+1} and v_{n+1/2} (and f_n); kick_kernel / unkick_kernel convert from /
// to the whole-step state q_n, v_n at the API boundary.
//   facet_kernel   per facet: rigid-body jump and strain (Sec. 2, Eq. (1)), per-tetrahedron
//                  volumetric strain (App. A.2 e_V), the Appendix A law, force A P t; then per
//                  tetrahedron vertex the fixed-order sum of its 6 facets' forces and moments
//                  (the tetrahedron's share of Eq. (2a)-(2b));
//   gather_kernel  per particle: fixed-order sum of its (tetrahedron, vertex) shares, then the second
//                  half kick of this step, the energy increments, and the first half kick and drift
//                  of the next step.
// The pass is bound by HBM bandwidth: no tensor cores (no dense contraction), no float atomics.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#include "ldpm_internal.h"

namespace ldpm {
namespace {

constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------------------------------------------
// Small vector helpers.
// ------------------------------------------------------------------------------------------------
template <class R>
struct V3 {
    R x, y, z;
};
template <class R>
__device__ __forceinline__ V3<R> operator-(V3<R> a, V3<R> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class R>
__device__ __forceinline__ V3<R> operator+(V3<R> a, V3<R> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class R>
__device__ __forceinline__ V3<R> operator*(R s, V3<R> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class R>
__device__ __forceinline__ R dot(V3<R> a, V3<R> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class R>
__device__ __forceinline__ V3<R> cross(V3<R> a, V3<R> b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

__device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }

// Exponentials of the facet law.  FP64 mode: the library functions.  Mixed mode: the hardware
// approximations (exp via ex2, x^y via lg2/ex2; errors of a few ulp, far inside the mixed-mode
// tolerances).  This translation unit is compiled with approximate FP32 division and square root
// (-prec-div=false -prec-sqrt=false), which touches only the mixed-mode arithmetic.
__device__ __forceinline__ float exp_(float x) { return __expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
// x^y for x >= 0, y >= 0
__device__ __forceinline__ float powpos_(float x, float y)
{
    return x > 0.0f ? exp2f(y * __log2f(x)) : (y == 0.0f ? 1.0f : 0.0f);
}
__device__ __forceinline__ double powpos_(double x, double y) { return pow(x, y); }

// Tangent pair (m, l) of a unit normal n: the branch-free orthonormal basis of Duff et al.,
// "Building an Orthonormal Basis, Revisited" (JCGT 6(1), 2017).  Any orthonormal tangents are
// allowed (paper Sec. 2); this choice is continuous except across n_z = 0.
template <class R>
__device__ __forceinline__ void tangent_frame(V3<R> n, V3<R> &m, V3<R> &l)
{
    const R sgn = copysign(R(1), n.z);
    const R a = R(-1) / (sgn + n.z);
    const R b = n.x * n.y * a;
    m = {R(1) + sgn * n.x * n.x * a, sgn * b, -sgn * n.x};
    l = {b, sgn + n.y * n.y * a, -n.y};
}

// ------------------------------------------------------------------------------------------------
// Appendix A constitutive update of one facet.  e: strain, de: its increment over this step, eV:
// volumetric strain of the tetrahedron, l: facet (edge) length; t/emax: previous history in,
// new history out.
// ------------------------------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void facet_law(const LawConst<R> &c, R l, V3<R> e, V3<R> de, R eV, R &tN, R &tM,
                                          R &tL, R &emax)
{
    const R E0 = c.E0, alpha = c.alpha;
    if (c.elastic) {  // Sec. 2: t = E0 diag(1, alpha, alpha) e
        tN = E0 * e.x;
        tM = alpha * E0 * e.y;
        tL = alpha * E0 * e.z;
        return;
    }
    if (e.x > R(0)) {
        // App. A.1 fracture.  Effective strain, coupling angle omega (sin = e_N / e,
        // cos = sqrt(alpha e_T^2) / e), strength sigma_0(omega) written as
        // 2 sigma_t / (sin + sqrt(sin^2 + 4 alpha cos^2 / r_st^2)) (the paper's expression with
        // numerator and denominator multiplied by the conjugate; finite at omega = pi/2).
        const R aT2 = alpha * (e.y * e.y + e.z * e.z);
        const R eeff = sqrt(e.x * e.x + aT2);
        if (eeff < c.tiny_strain) {
            // t / e is 0/0 at vanishing strain (its squares underflow first); the elastic limit
            // t = E e applies.  Reached ahead of a loading wave, where strains decay to ~0.
            tN = E0 * e.x;
            tM = alpha * E0 * e.y;
            tL = alpha * E0 * e.z;
            emax = emax > eeff ? emax : eeff;
            return;
        }
        const R saT = sqrt(aT2);
        const R omega = atan2(e.x, saT);
        const R inv_e = R(1) / eeff;
        const R sn = e.x * inv_e, cs = saT * inv_e;
        const R sigma0 = R(2) * c.sigma_t / (sn + sqrt(sn * sn + c.four_alpha_over_r2 * cs * cs));
        // H_t = 2 E0 / (l_t / l - 1) = 2 E0 l / (l_t - l); H_0 = H_s/alpha + (H_t - H_s/alpha)(2 omega/pi)^n_t
        const R Ht = R(2) * E0 * l / (c.l_t - l);
        const R H0 = c.Hs_over_alpha + (Ht - c.Hs_over_alpha) * powpos_(omega * R(2.0 / kPi), c.n_t);
        const R e0 = sigma0 / E0;
        emax = emax > eeff ? emax : eeff;
        const R over = emax - e0 > R(0) ? emax - e0 : R(0);
        const R sigma_bt = sigma0 * exp_(-H0 * over / sigma0);
        // t = t_old + E0 (e - e_old).  The effective-strain difference is formed from the increment:
        // e^2 - e_old^2 = sum_i w_i de_i (2 e_i - de_i) with w = (1, alpha, alpha), divided by
        // (e + e_old) -- algebraically the same, free of the cancellation of two nearby roots.
        const V3<R> ep = e - de;
        const R e_old = sqrt(ep.x * ep.x + alpha * (ep.y * ep.y + ep.z * ep.z));
        const R num = de.x * (e.x + ep.x) + alpha * (de.y * (e.y + ep.y) + de.z * (e.z + ep.z));
        const R d_eff = num / (eeff + e_old);
        const R t_old = sqrt(tN * tN + (tM * tM + tL * tL) * c.inv_alpha);
        R t = t_old + E0 * d_eff;
        t = t < R(0) ? R(0) : t;
        t = t > sigma_bt ? sigma_bt : t;
        const R r = t * inv_e;
        tN = r * e.x;
        tM = alpha * r * e.y;
        tL = alpha * r * e.z;
        return;
    }
    // App. A.2 compression: t_N incrementally elastic (E_Nc), -sigma_bc <= t_N <= 0.
    const R ENc = (-tN <= c.sigma_c0) ? E0 : c.Ed;
    R tn = tN + ENc * de.x;
    const R eD = e.x - eV;
    const R eDV = eV + c.beta * eD;
    const R rDV = (eV <= R(0)) ? -fabs(eD) / (eV - c.eV0) : fabs(eD) / c.eV0;
    const R mac = rDV - c.kc1 > R(0) ? rDV - c.kc1 : R(0);
    const R Hc = (c.Hc0 - c.Hc1) / (R(1) + c.kc2 * mac) + c.Hc1;
    R sigma_bc;
    if (-eDV <= R(0)) {
        sigma_bc = c.sigma_c0;
    } else if (-eDV <= c.ec1) {
        const R o = -eDV - c.ec0 > R(0) ? -eDV - c.ec0 : R(0);
        sigma_bc = c.sigma_c0 + o * Hc;
    } else {
        const R sigma_c1 = c.sigma_c0 + (c.ec1 - c.ec0) * Hc;
        sigma_bc = sigma_c1 * exp_((-eDV - c.ec1) * Hc / sigma_c1);
    }
    tn = tn < -sigma_bc ? -sigma_bc : tn;
    tn = tn > R(0) ? R(0) : tn;
    // App. A.3 friction: elastic shear trial, radial return onto sqrt(t_M^2 + t_L^2) = sigma_bs(t_N).
    R tm = tM + alpha * E0 * de.y;
    R tl = tL + alpha * E0 * de.z;
    const R sigma_bs = c.sigma_s + c.mu_diff_sN0 - c.mu_inf * tn - c.mu_diff_sN0 * exp_(tn * c.inv_sigma_N0);
    const R tau2 = tm * tm + tl * tl;
    if (tau2 > sigma_bs * sigma_bs) {
        const R s = sigma_bs * rsqrt_(tau2);
        tm *= s;
        tl *= s;
    }
    tN = tn;
    tM = tm;
    tL = tl;
}

// ------------------------------------------------------------------------------------------------
// Facet pass.  A block owns TETS consecutive tetrahedra (12 * TETS facets, one thread each).
//   phase A  4 threads per tetrahedron gather the vertex records (mixed mode: the 96-byte FP32
//            mirror, two-float differences; FP64 mode: the 128-byte FP64 record) and write the
//            differences to vertex 0 of the tetrahedron to shared memory, then the tetrahedron's
//            volumetric strain;
//   phase B  one thread per facet: kinematics, law, force, and its contributions to its two
//            vertices (force and moment about each);
//   phase C  12 threads per tetrahedron: thread s sums components 2(s%3), 2(s%3)+1 of vertex s/3
//            over the vertex's 6 facets in a fixed order (its 3 edges ascending, each edge's two
//            facets in slot order).
// Shared-memory rows are 16-byte aligned and accessed with 128/64-bit vectors (the pass is bound by
// L1/shared-memory wavefronts before HBM).  The facet's geometry and history are loaded into
// registers before phase A so their HBM latency overlaps the gathers.
// ------------------------------------------------------------------------------------------------
constexpr int kRow = 16;  // vertex row: dx(3) du(3) dv(3) theta(3) omega(3) pad
constexpr int kCon = 12;  // facet row: contribution to vertex a (6), to vertex b (6)
// Row strides in elements: with 16-byte accesses, 8 consecutive rows must start in distinct 4-bank
// groups (stride = 4 mod 8 banks for floats is 20 or 12 words; doubles use 36 and 28 words).
template <class R>
struct Stride {
    static constexpr int row = sizeof(R) == 4 ? 20 : 18;
    static constexpr int con = sizeof(R) == 4 ? 12 : 14;
};

template <class R>
struct VecT;
template <>
struct VecT<float> {
    using v16 = float4;  // 16-byte vector
    using v2 = float2;   // pair
    static __device__ __forceinline__ void put(float *d, const float *s) { *reinterpret_cast<float4 *>(d) = float4{s[0], s[1], s[2], s[3]}; }
    static __device__ __forceinline__ void get(float *d, const float *s)
    {
        const float4 w = *reinterpret_cast<const float4 *>(s);
        d[0] = w.x;
        d[1] = w.y;
        d[2] = w.z;
        d[3] = w.w;
    }
};
template <>
struct VecT<double> {
    using v16 = double2;
    using v2 = double2;
    static __device__ __forceinline__ void put(double *d, const double *s) { *reinterpret_cast<double2 *>(d) = double2{s[0], s[1]}; }
    static __device__ __forceinline__ void get(double *d, const double *s)
    {
        const double2 w = *reinterpret_cast<const double2 *>(s);
        d[0] = w.x;
        d[1] = w.y;
    }
};

template <class R, int MODE, int TETS>
__global__ void __launch_bounds__(12 * TETS) facet_kernel(DeviceModel m, const void *__restrict__ vsrc)
{
    using T4 = R4<R>;
    using V2 = typename VecT<R>::v2;
    constexpr int E = 16 / (int)sizeof(R);  // elements per 16-byte shared-memory vector
    __shared__ alignas(16) R sv[TETS * 4][Stride<R>::row];
    __shared__ alignas(16) R scon[12 * TETS][Stride<R>::con];
    __shared__ R seV[TETS];
    __shared__ int sok[TETS];
    const T4 *__restrict__ geo = static_cast<const T4 *>(m.geo);
    T4 *__restrict__ hist = static_cast<T4 *>(m.hist);
    T4 *__restrict__ fout = static_cast<T4 *>(m.fout);
    R *__restrict__ tvc = static_cast<R *>(m.tvc);
    const LawConst<R> *__restrict__ lawc = static_cast<const LawConst<R> *>(m.law);

    const int tid = threadIdx.x;
    const int64_t tet0 = (int64_t)blockIdx.x * TETS;
    if (MODE == FACET_STEP && blockIdx.x == 0 && tid == 0) *m.step += 1;

    // ---- prefetch this thread's facet data
    const int j = tid / 12;
    const int slot = tid - 12 * j;
    const int64_t f = tet0 * 12 + tid;
    const bool valid = tet0 + j < m.T;
    T4 g{}, h{};
    if (valid) {
        g = geo[f];
        if (MODE != FACET_ELASTIC) h = hist[f];
    }

    // ---- phase A: vertex records -> shared memory, e_V per tetrahedron
    if (tid < 4 * TETS) {
        const int jt = tid >> 2, vi = tid & 3;
        const int64_t tt = tet0 + jt;
        int p = -1;
        if (tt < m.T) p = reinterpret_cast<const int *>(m.tet)[4 * tt + vi];
        const int base = (threadIdx.x & 31) & ~3;
        R o[kRow];
        if constexpr (sizeof(R) == 4) {
            // mirror: x_hi 0..2, x_lo 3..5, u_hi 6..8, u_lo 9..11, theta 12..14, v 15..17, omega 18..20.
            // (a_hi - b_hi) + (a_lo - b_lo) carries FP32 relative accuracy of the difference itself.
            const float *src = static_cast<const float *>(vsrc);
            float rec[24];
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
            } else {
#pragma unroll
                for (int k = 0; k < 24; ++k) rec[k] = 0.0f;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float x0h = __shfl_sync(0xffffffffu, rec[k], base);
                const float x0l = __shfl_sync(0xffffffffu, rec[3 + k], base);
                const float u0h = __shfl_sync(0xffffffffu, rec[6 + k], base);
                const float u0l = __shfl_sync(0xffffffffu, rec[9 + k], base);
                const float v0 = __shfl_sync(0xffffffffu, rec[15 + k], base);
                o[k] = (rec[k] - x0h) + (rec[3 + k] - x0l);
                o[3 + k] = (rec[6 + k] - u0h) + (rec[9 + k] - u0l);
                o[6 + k] = rec[15 + k] - v0;
                o[9 + k] = rec[12 + k];
                o[12 + k] = rec[18 + k];
            }
        } else {
            // FP64 record: x 0..2, u 3..5, theta 6..8, v 9..11, omega 12..14
            const double *src = static_cast<const double *>(vsrc);
            double rec[16];
            if (p >= 0) {
                const double2 *r2 = reinterpret_cast<const double2 *>(src + 16 * (int64_t)p);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const double2 w = r2[k];
                    rec[2 * k] = w.x;
                    rec[2 * k + 1] = w.y;
                }
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) rec[k] = 0.0;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double x0 = __shfl_sync(0xffffffffu, rec[k], base);
                const double u0 = __shfl_sync(0xffffffffu, rec[3 + k], base);
                const double v0 = __shfl_sync(0xffffffffu, rec[9 + k], base);
                o[k] = rec[k] - x0;
                o[3 + k] = rec[3 + k] - u0;
                o[6 + k] = rec[9 + k] - v0;
                o[9 + k] = rec[6 + k];
                o[12 + k] = rec[12 + k];
            }
        }
        if (MODE == FACET_METRIC) {  // whole-step state: u_n = u_{n+1} - dt v_{n+1/2}, same for theta
            const R dtm = lawc[m.tile_spec ? m.tile_spec[tet0 / 32] : 0].dt;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                o[3 + k] -= dtm * o[6 + k];
                o[9 + k] -= dtm * o[12 + k];
            }
        }
        o[15] = R(0);
#pragma unroll
        for (int k = 0; k < kRow; k += E) VecT<R>::put(&sv[tid][k], &o[k]);
        // e_V = (1/3) div u of the linear tetrahedron.  With D = [dx1 dx2 dx3], grad N_i (i = 1..3)
        // are the rows of D^-1 = [dx2 x dx3; dx3 x dx1; dx1 x dx2] / det D, and vertex 0 carries no
        // displacement difference.  Lane i >= 1 forms its own term du_i . (dx_i1 x dx_i2).
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
        const V3<R> cr = cross(a1, a2);
        R term = vi == 0 ? R(0) : dot(dus, cr);
        R det = vi == 0 ? R(0) : dot(dxs, cr);
        term += __shfl_xor_sync(0xffffffffu, term, 1);
        term += __shfl_xor_sync(0xffffffffu, term, 2);
        det = __shfl_sync(0xffffffffu, det, base + 1);
        if (vi == 0) {
            seV[jt] = (p >= 0 && det != R(0)) ? term / (R(3) * det) : R(0);
            sok[jt] = p >= 0;
        }
    }
    __syncthreads();

    // ---- phase B: one facet
    const bool live = valid && sok[j];
    R cs[12];
    if (!live) {
#pragma unroll
        for (int k = 0; k < 12; ++k) cs[k] = R(0);
    } else {
        const int e = slot >> 1;
        const int va = (0x211000 >> (4 * e)) & 0xF;
        const int vb = (0x332321 >> (4 * e)) & 0xF;
        R A[kRow], B[kRow];
#pragma unroll
        for (int k = 0; k < kRow; k += E) {
            VecT<R>::get(&A[k], &sv[4 * j + va][k]);
            VecT<R>::get(&B[k], &sv[4 * j + vb][k]);
        }
        const V3<R> d = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        const R inv_l = rsqrt_(dot(d, d));
        const R l = dot(d, d) * inv_l;
        const V3<R> n = inv_l * d;
        V3<R> mt, lt;
        tangent_frame(n, mt, lt);
        const V3<R> ca = {g.x, g.y, g.z};
        const V3<R> cb = ca - d;
        R tN, tM, tL, emax;
        const int sp = m.tile_spec ? m.tile_spec[tet0 / 32] : 0;  // specimens are padded to 32 tetrahedra
        const LawConst<R> &c = lawc[sp];
        if (MODE == FACET_FROM_HIST) {
            tN = h.x;
            tM = h.y;
            tL = h.z;
        } else {
            const V3<R> thA = {A[9], A[10], A[11]}, thB = {B[9], B[10], B[11]};
            const V3<R> du = {B[3] - A[3], B[4] - A[4], B[5] - A[5]};
            const V3<R> jump = du + cross(thB, cb) - cross(thA, ca);
            const V3<R> e3 = {dot(n, jump) * inv_l, dot(mt, jump) * inv_l, dot(lt, jump) * inv_l};
            if (MODE == FACET_ELASTIC) {
                tN = c.E0 * e3.x;
                tM = c.alpha * c.E0 * e3.y;
                tL = c.alpha * c.E0 * e3.z;
            } else if (MODE == FACET_METRIC) {
                // crack opening from the inelastic part of the jump: w_N = l <e_N - t_N / E0>,
                // w_T = l (e_T - t_T / (alpha E0)) (u here is already u_n)
                R wn = e3.x - h.x / c.E0;
                wn = wn > R(0) ? wn : R(0);
                const R aE = c.alpha * c.E0;
                const R wm = e3.y - h.y / aE, wl = e3.z - h.z / aE;
                T4 o4;
                o4.x = l * sqrt(wn * wn + wm * wm + wl * wl);
                o4.y = seV[j];
                o4.z = R(0);
                o4.w = R(0);
                fout[f] = o4;
                tN = tM = tL = R(0);
            } else {
                const V3<R> omA = {A[12], A[13], A[14]}, omB = {B[12], B[13], B[14]};
                const V3<R> dv = {B[6] - A[6], B[7] - A[7], B[8] - A[8]};
                const V3<R> djump = dv + cross(omB, cb) - cross(omA, ca);
                const R sdt = c.dt * inv_l;
                const V3<R> de3 = {dot(n, djump) * sdt, dot(mt, djump) * sdt, dot(lt, djump) * sdt};
                tN = h.x;
                tM = h.y;
                tL = h.z;
                emax = h.w;
                facet_law(c, l, e3, de3, seV[j], tN, tM, tL, emax);
                T4 hn;
                hn.x = tN;
                hn.y = tM;
                hn.z = tL;
                hn.w = emax;
                hist[f] = hn;
            }
        }
        const R Ar = g.w;
        const V3<R> F = {Ar * (tN * n.x + tM * mt.x + tL * lt.x), Ar * (tN * n.y + tM * mt.y + tL * lt.y),
                         Ar * (tN * n.z + tM * mt.z + tL * lt.z)};
        if (MODE == FACET_FROM_HIST) {  // per-facet force, kept only for ldpm_facet_forces
            T4 Fo;
            Fo.x = F.x;
            Fo.y = F.y;
            Fo.z = F.z;
            Fo.w = R(0);
            fout[f] = Fo;
        }
        // vertex a receives +F and the moment c_a x F about itself; vertex b -F and c_b x (-F)
        const V3<R> Ma = cross(ca, F);
        const V3<R> Mb = cross(cb, F);
        cs[0] = F.x;
        cs[1] = F.y;
        cs[2] = F.z;
        cs[3] = Ma.x;
        cs[4] = Ma.y;
        cs[5] = Ma.z;
        cs[6] = -F.x;
        cs[7] = -F.y;
        cs[8] = -F.z;
        cs[9] = -Mb.x;
        cs[10] = -Mb.y;
        cs[11] = -Mb.z;
    }
#pragma unroll
    for (int k = 0; k < kCon; k += E) VecT<R>::put(&scon[tid][k], &cs[k]);
    __syncthreads();

    // ---- phase C: thread `slot` of tetrahedron j sums components 2 q, 2 q + 1 (q = slot % 3) of
    // vertex v = slot / 3 over its 3 edges (ascending), each edge's two facets in slot order.
    if (live && MODE != FACET_METRIC) {
        const int v = slot / 3;
        const int q = slot - 3 * v;
        const int edges = (int)((0x542531430210ull >> (12 * v)) & 0xFFF);
        const int sides = (0xEC8 >> (3 * v)) & 0x7;  // v0: 000, v1: 001, v2: 011, v3: 111
        R s0 = R(0), s1 = R(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int e2 = (edges >> (4 * k)) & 0xF;
            const int col = (((sides >> k) & 1) ? 6 : 0) + 2 * q;
            const V2 w0 = *reinterpret_cast<const V2 *>(&scon[12 * j + 2 * e2][col]);
            const V2 w1 = *reinterpret_cast<const V2 *>(&scon[12 * j + 2 * e2 + 1][col]);
            s0 += w0.x;
            s1 += w0.y;
            s0 += w1.x;
            s1 += w1.y;
        }
        *reinterpret_cast<V2 *>(tvc + (tet0 + j) * 24 + 6 * v + 2 * q) = V2{s0, s1};
    }
}

// ------------------------------------------------------------------------------------------------
// Particle pass.  A group of LPP lanes owns one particle: it sums the particle's (tetrahedron,
// vertex) contributions in CSR order (Eq. (2a)-(2b)), reduces across the group, and lanes 0..5 of the
// group update one DOF each.  In mixed mode the contributions are FP32 values and their sums are
// formed in FP32 (this adds rounding of the same order as the forces' own); everything after the sum
// is FP64.  With LPP = 8 a
// warp updates 4 particles per FP64 instruction: the GB300 FP64 pipe issues one warp instruction
// per ~64 cycles per sub-partition, so FP64 instruction count, not bytes, bounds this pass if the
// whole warp serves one particle.
// ------------------------------------------------------------------------------------------------
// ramp(t) = clamp(t / T, 0, 1), given invT = 1/T (invT = 0: no ramp, ramp = 1)
__device__ __forceinline__ double ramp(double t, double invT)
{
    if (invT == 0.0) return 1.0;
    const double r = t * invT;
    return r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
}


// Finite test on the exponent bits (integer pipe).
__device__ __forceinline__ bool finite_bits(double x)
{
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// IEEE-754 conversions done with integer instructions.  The GB300 FP64 pipe (which also executes
// F2F conversions) issues one warp instruction per ~64 cycles per sub-partition; these bit
// manipulations run at integer rate.  Magnitudes below the normal float range become signed zeros
// (|x| < 1.2e-38 in mm, N or rad: never significant for the facet pass).
__device__ __forceinline__ float d2f_trunc(double x)  // mantissa truncated: error < 1 float ulp
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int eb = (int)((b >> 52) & 0x7ff);
    const int e = eb - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) {  // overflow -> inf; NaN stays NaN
        const bool nan = eb == 0x7ff && (b & 0xfffffffffffffull) != 0;
        return __uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u));
    }
    return __uint_as_float(sign | ((uint32_t)e << 23) | (uint32_t)((b >> 29) & 0x7fffffu));
}

// x = hi + lo: hi the truncated float of x, lo the truncated float of the 29 dropped mantissa bits
// (relative error of hi + lo below 2^-46).
__device__ __forceinline__ void d2f_split(double x, float &hi, float &lo)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int eb = (int)((b >> 52) & 0x7ff);
    const int e = eb - 1023 + 127;
    if (e <= 0 || e >= 255) {
        hi = d2f_trunc(x);
        lo = 0.0f;
        return;
    }
    hi = __uint_as_float(sign | ((uint32_t)e << 23) | (uint32_t)((b >> 29) & 0x7fffffu));
    const uint32_t rem = (uint32_t)(b & 0x1fffffffu);  // value rem * 2^(eb - 1075)
    const int lz = __clz(rem);                         // 32 when rem == 0
    const int fe = (31 - lz) + eb - 1075 + 127;        // float exponent of the remainder
    if (rem == 0 || fe <= 0) {
        lo = 0.0f;
        return;
    }
    const uint32_t frac = ((uint32_t)((uint64_t)rem << (lz + 1))) >> 9;  // leading one dropped
    lo = __uint_as_float(sign | ((uint32_t)fe << 23) | frac);
}

// float -> double (exact for normal floats; float denormals become signed zeros).
__device__ __forceinline__ double f2d_bits(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0) return __longlong_as_double((long long)sign);
    const uint64_t ed = e == 255 ? 0x7ffull : (uint64_t)(e + 896);
    return __longlong_as_double((long long)(sign | (ed << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
}

// FP32 mirror entries of DOF d of a particle after its FP64 q and v changed.
__device__ __forceinline__ void write_mirror(float *pm, int d, double q, double v)
{
    if (d < 3) {
        float hi, lo;
        d2f_split(q, hi, lo);
        pm[6 + d] = hi;
        pm[9 + d] = lo;
        pm[15 + d] = d2f_trunc(v);
    } else {
        pm[12 + d - 3] = d2f_trunc(q);
        pm[18 + d - 3] = d2f_trunc(v);
    }
}

template <class R>
__device__ __forceinline__ double to_double(R x)
{
    if constexpr (sizeof(R) == 4)
        return f2d_bits(x);
    else
        return x;
}

template <class R, int MODE, int LPP>
__global__ void __launch_bounds__(256) gather_kernel(DeviceModel m, double *__restrict__ out6)
{
    static_assert(LPP == 8 || LPP == 16 || LPP == 32, "lanes per particle");
    using R2 = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
    const int32_t *__restrict__ ent = static_cast<const int32_t *>(m.ent);
    const R *__restrict__ tvc = static_cast<const R *>(m.tvc);
    const int lane = threadIdx.x & 31;
    const int sub = lane & (LPP - 1);
    const int64_t p = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / LPP) + lane / LPP;
    const bool valid = p < m.N;
    int r0 = 0, r1 = 0;
    if (valid) {
        r0 = m.row[p];
        r1 = m.row[p + 1];
    }
    // each entry is one (tetrahedron, vertex) slot: 6 values, force (3) and moment about the particle (3)
    R a[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    for (int r = r0 + sub; r < r1; r += 2 * LPP) {
        int id[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) id[k] = (r + k * LPP < r1) ? ent[r + k * LPP] : -1;
        R2 w[2][3];
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (id[k] >= 0) {
                const R2 *src = reinterpret_cast<const R2 *>(tvc + 6 * (int64_t)id[k]);
                w[k][0] = src[0];
                w[k][1] = src[1];
                w[k][2] = src[2];
            }
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (id[k] >= 0) {
                a[0] += w[k][0].x;
                a[1] += w[k][0].y;
                a[2] += w[k][1].x;
                a[3] += w[k][1].y;
                a[4] += w[k][2].x;
                a[5] += w[k][2].y;
            }
    }
#pragma unroll
    for (int off = LPP / 2; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < 6; ++k) a[k] += __shfl_xor_sync(0xffffffffu, a[k], off);
    // lanes 0..5 of the group own one DOF each; the other lanes mirror DOF 0 and store nothing
    const bool act = valid && sub < 6;
    const int d = sub < 6 ? sub : 0;
    R fr = a[0];
#pragma unroll
    for (int k = 1; k < 6; ++k)
        if (d == k) fr = a[k];
    const double fa_new = to_double<R>(fr);
    if (MODE == GATHER_ASSEMBLE) {
        if (act) out6[6 * p + d] = fa_new;
        return;
    }
    // ---- velocity-form central difference for DOF d (state on entry: q_{n+1}, v_{n+1/2}, f_n)
    const int64_t pc_ = valid ? p : 0;
    double *ps = m.pstate + 16 * pc_;
    double *pd = m.pdyn + 8 * pc_;
    const double *pc = m.pconst + 8 * pc_;
    const double im = pc[d];
    const uint64_t bcbits = (uint64_t)__double_as_longlong(pc[6]);
    const int mask = (int)((bcbits >> (8 * d)) & 0xffu);
    const int sp = (int)__double_as_longlong(pc[7]);
    const SpecDyn &S = m.spec[sp];
    const double dt = S.dt, hdt = S.half_dt;
    const bool has_fext = m.f_ext != nullptr;
    const double fe = has_fext ? m.f_ext[6 * pc_ + d] : 0.0;
    const double vh = ps[9 + d];
    const double fa_old = pd[d];
    // energy terms need the external work only where a lane is constrained or loaded
    const bool need_we = __any_sync(0xffffffffu, act && (mask != 0 || has_fext));
    double g_sum = 0.0, v_new, v_next;
    if (mask == 0) {
        const double dv = (has_fext ? fe + fa_new : fa_new) * (hdt * im);  // dt/2 a_{n+1}
        if (has_fext) g_sum = 2.0 * fe;
        v_new = vh + dv;
        v_next = v_new + dv;
    } else if (mask == 1) {
        g_sum = -(fa_old + fa_new);
        v_new = 0.0;
        v_next = 0.0;
    } else {
        // prescribed velocity vb ramp(t); the constraint's accelerations at t_n and t_{n+1} are
        // vb (ramp(t +- dt/2) differences) / dt, so their sum telescopes to vb (r(t1+dt/2) - r(t0-dt/2)) / dt
        const int64_t n1 = *m.step;
        const double t1 = (double)n1 * dt;
        const double vb = m.bc_vel[6 * pc_ + d];
        const double r_next = ramp(t1 + hdt, S.inv_ramp);
        g_sum = m.bc_vm[6 * pc_ + d] * (r_next - ramp(t1 - dt - hdt, S.inv_ramp)) * S.inv_dt - (fa_old + fa_new);
        v_new = vb * ramp(t1, S.inv_ramp);
        v_next = vb * r_next;
    }
    // energy increments over [t_n, t_{n+1}] (trapezoid): dq = dt v_{n+1/2}
    const double hdq = hdt * vh;
    double dWi = act ? -(fa_old + fa_new) * hdq : 0.0;
    double dWe = (need_we && act) ? g_sum * hdq : 0.0;
    // store the drifted state of the next step: v_{n+3/2} and q_{n+2} = q_{n+1} + dt v_{n+3/2}
    (void)v_new;
    const double v_store = v_next;
    const double q = ps[3 + d] + dt * v_next;
    // sum the six DOF contributions into lane 0 of the group (lanes 6, 7 hold zeros)
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) dWi += __shfl_xor_sync(0xffffffffu, dWi, off);
    if (need_we) {
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) dWe += __shfl_xor_sync(0xffffffffu, dWe, off);
    }
    if (act) {
        pd[d] = fa_new;
        ps[3 + d] = q;
        ps[9 + d] = v_store;
        if (m.pm32) write_mirror(m.pm32 + kMirror * pc_, d, q, v_store);
        if (!finite_bits(v_store) || !finite_bits(q)) *(volatile int32_t *)m.flag = 1;
        if (sub == 0) {
            pd[6] += dWi;
            if (need_we) pd[7] += dWe;
        }
    }
}

// First half kick and drift of a stepping call: v_{n+1/2} = v_n + dt/2 a_n, q_{n+1} = q_n + dt v_{n+1/2}.
__global__ void __launch_bounds__(256) kick_kernel(DeviceModel m)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * (int64_t)m.N) return;
    const int64_t p = i / 6;
    const int d = (int)(i - 6 * p);
    double *ps = m.pstate + 16 * p;
    const double *pc = m.pconst + 8 * p;
    const int mask = (int)(((uint64_t)__double_as_longlong(pc[6]) >> (8 * d)) & 0xffu);
    const int sp = (int)__double_as_longlong(pc[7]);
    const double dt = m.spec[sp].dt;
    double vh;
    if (mask == 0) {
        const double fe = m.f_ext ? m.f_ext[6 * p + d] : 0.0;
        vh = ps[9 + d] + 0.5 * dt * (fe + m.pdyn[8 * p + d]) * pc[d];
    } else if (mask == 1) {
        vh = 0.0;
    } else {
        const double t = (double)(*m.step) * dt;
        vh = m.bc_vel[6 * p + d] * ramp(t + 0.5 * dt, m.spec[sp].inv_ramp);
    }
    const double q = ps[3 + d] + dt * vh;
    ps[9 + d] = vh;
    ps[3 + d] = q;
    if (m.pm32) write_mirror(m.pm32 + kMirror * p, d, q, vh);
}

// Whole-step state (q_n, v_n) from the drifted state (q_{n+1}, v_{n+1/2}) the library keeps between
// calls: the inverse of kick_kernel under the same boundary conditions.  out12 [N][12] (q then v),
// or null to rewrite pstate (and the mirror) in place.
__global__ void __launch_bounds__(256) unkick_kernel(DeviceModel m, double *__restrict__ out12)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * (int64_t)m.N) return;
    const int64_t p = i / 6;
    const int d = (int)(i - 6 * p);
    double *ps = m.pstate + 16 * p;
    const double *pc = m.pconst + 8 * p;
    const int mask = (int)(((uint64_t)__double_as_longlong(pc[6]) >> (8 * d)) & 0xffu);
    const SpecDyn &S = m.spec[(int)__double_as_longlong(pc[7])];
    const double vh = ps[9 + d];
    double vn;
    if (mask == 0) {
        const double fe = m.f_ext ? m.f_ext[6 * p + d] : 0.0;
        vn = vh - S.half_dt * (fe + m.pdyn[8 * p + d]) * pc[d];
    } else if (mask == 1) {
        vn = 0.0;
    } else {
        vn = m.bc_vel[6 * p + d] * ramp((double)(*m.step) * S.dt, S.inv_ramp);
    }
    const double qn = ps[3 + d] - S.dt * vh;
    if (out12) {
        out12[12 * p + d] = qn;
        out12[12 * p + 6 + d] = vn;
    } else {
        ps[3 + d] = qn;
        ps[9 + d] = vn;
        if (m.pm32) write_mirror(m.pm32 + kMirror * p, d, qn, vn);
    }
}

// FP32 mirror of every particle from the FP64 records.
__global__ void __launch_bounds__(256) mirror_kernel(DeviceModel m)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m.N) return;
    const double *ps = m.pstate + 16 * p;
    float *pm = m.pm32 + kMirror * p;
    for (int k = 0; k < 3; ++k) d2f_split(ps[k], pm[k], pm[3 + k]);
    for (int d = 0; d < 6; ++d) write_mirror(pm, d, ps[3 + d], ps[9 + d]);
    for (int k = 21; k < kMirror; ++k) pm[k] = 0.0f;
}

// Energy sums over particles [p0, p1) (per block, fixed order), then one block adds the partials.
__global__ void __launch_bounds__(256) energy_kernel(DeviceModel m, int32_t p0, int32_t p1, double *partial)
{
    __shared__ double red[256][16];
    const int tid = threadIdx.x;
    const int64_t p = (int64_t)p0 + (int64_t)blockIdx.x * 256 + tid;
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    if (p < p1) {
        const double *ps = m.pstate + 16 * p;
        const double *pd = m.pdyn + 8 * p;
        const double *pc = m.pconst + 8 * p;
        const uint64_t bcbits = (uint64_t)__double_as_longlong(pc[6]);
        const int sp = (int)__double_as_longlong(pc[7]);
        const SpecDyn &S = m.spec[sp];
        const double dt = S.dt;
        const double t = (double)(*m.step) * dt;
        acc[0] = pd[6];
        acc[1] = pd[7];
        for (int d = 0; d < 6; ++d) {
            const double mass = 1.0 / pc[d];
            // whole-step velocity v_n from the stored v_{n+1/2} (inverse half kick)
            const int mk = (int)((bcbits >> (8 * d)) & 0xffu);
            double v = ps[9 + d];
            if (mk == 0)
                v -= S.half_dt * ((m.f_ext ? m.f_ext[6 * p + d] : 0.0) + pd[d]) * pc[d];
            else if (mk == 1)
                v = 0.0;
            else
                v = m.bc_vel[6 * p + d] * ramp(t, S.inv_ramp);
            acc[2] += 0.5 * mass * v * v;
            const int mask = (int)((bcbits >> (8 * d)) & 0xffu);
            if (mask == 1) {
                acc[4 + d] += -pd[d];
            } else if (mask == 2) {
                const double ra = ramp(t + 0.5 * dt, S.inv_ramp) - ramp(t - 0.5 * dt, S.inv_ramp);
                acc[10 + d] += m.bc_vm[6 * p + d] * ra * S.inv_dt - pd[d];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) red[tid][k] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w)
#pragma unroll
            for (int k = 0; k < 16; ++k) red[tid][k] += red[tid + w][k];
        __syncthreads();
    }
    if (tid < 16) partial[16 * (int64_t)blockIdx.x + tid] = red[0][tid];
}

__global__ void __launch_bounds__(256) energy_final_kernel(const double *partial, int32_t nb, double *out16)
{
    __shared__ double red[256][16];
    const int tid = threadIdx.x;
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    for (int b = tid; b < nb; b += 256)
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] += partial[16 * (int64_t)b + k];
#pragma unroll
    for (int k = 0; k < 16; ++k) red[tid][k] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w)
#pragma unroll
            for (int k = 0; k < 16; ++k) red[tid][k] += red[tid + w][k];
        __syncthreads();
    }
    if (tid < 16) out16[tid] = red[0][tid];
}

// History <-> caller format (t_N, global tangential traction, e_max), in the internal facet order.
// The frame is rebuilt from the particle positions exactly as the facet pass forms it.
template <class R>
__device__ __forceinline__ bool facet_frame_of(const DeviceModel &m, int64_t f, V3<R> &n, V3<R> &mt, V3<R> &lt)
{
    const int64_t tt = f / 12;
    const int e = (int)(f - 12 * tt) >> 1;
    const int va = (0x211000 >> (4 * e)) & 0xF;
    const int vb = (0x332321 >> (4 * e)) & 0xF;
    const int *tv = reinterpret_cast<const int *>(m.tet) + 4 * tt;
    const int p0 = tv[0], pa = tv[va], pb = tv[vb];
    if (p0 < 0) return false;
    V3<R> dxa, dxb;
    if constexpr (sizeof(R) == 4) {
        const float *x0 = m.pm32 + kMirror * (int64_t)p0, *xa = m.pm32 + kMirror * (int64_t)pa,
                    *xb = m.pm32 + kMirror * (int64_t)pb;
        dxa = {(xa[0] - x0[0]) + (xa[3] - x0[3]), (xa[1] - x0[1]) + (xa[4] - x0[4]),
               (xa[2] - x0[2]) + (xa[5] - x0[5])};
        dxb = {(xb[0] - x0[0]) + (xb[3] - x0[3]), (xb[1] - x0[1]) + (xb[4] - x0[4]),
               (xb[2] - x0[2]) + (xb[5] - x0[5])};
    } else {
        const double *x0 = m.pstate + 16 * (int64_t)p0, *xa = m.pstate + 16 * (int64_t)pa,
                     *xb = m.pstate + 16 * (int64_t)pb;
        dxa = {R(xa[0] - x0[0]), R(xa[1] - x0[1]), R(xa[2] - x0[2])};
        dxb = {R(xb[0] - x0[0]), R(xb[1] - x0[1]), R(xb[2] - x0[2])};
    }
    const V3<R> d = dxb - dxa;
    const R inv_l = rsqrt_(dot(d, d));
    n = inv_l * d;
    tangent_frame(n, mt, lt);
    return true;
}

template <class R>
__global__ void hist_to_user_kernel(DeviceModel m, double *__restrict__ out5)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= 12 * (int64_t)m.T) return;
    V3<R> n, mt, lt;
    const R4<R> h = static_cast<const R4<R> *>(m.hist)[f];
    double *o = out5 + 5 * f;
    if (!facet_frame_of<R>(m, f, n, mt, lt)) {
        for (int k = 0; k < 5; ++k) o[k] = 0.0;
        return;
    }
    o[0] = double(h.x);
    o[1] = double(h.y) * double(mt.x) + double(h.z) * double(lt.x);
    o[2] = double(h.y) * double(mt.y) + double(h.z) * double(lt.y);
    o[3] = double(h.y) * double(mt.z) + double(h.z) * double(lt.z);
    o[4] = double(h.w);
}

template <class R>
__global__ void hist_from_user_kernel(DeviceModel m, const double *__restrict__ in5)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= 12 * (int64_t)m.T) return;
    V3<R> n, mt, lt;
    R4<R> h;
    h.x = h.y = h.z = h.w = R(0);
    if (facet_frame_of<R>(m, f, n, mt, lt)) {
        const double *u = in5 + 5 * f;
        h.x = R(u[0]);
        h.y = R(u[1] * double(mt.x) + u[2] * double(mt.y) + u[3] * double(mt.z));
        h.z = R(u[1] * double(lt.x) + u[2] * double(lt.y) + u[3] * double(lt.z));
        h.w = R(u[4]);
    }
    static_cast<R4<R> *>(m.hist)[f] = h;
}

template <class R, int MODE>
cudaError_t launch_facet_tpb(const DeviceModel &m, const void *pst, cudaStream_t s)
{
    const int tpb = m.tets_per_block;
    const unsigned blocks = (unsigned)((m.T + tpb - 1) / tpb);
    if (blocks == 0) return cudaSuccess;
    switch (tpb) {
    case 16:
        facet_kernel<R, MODE, 16><<<blocks, 192, 0, s>>>(m, pst);
        break;
    case 32:
        facet_kernel<R, MODE, 32><<<blocks, 384, 0, s>>>(m, pst);
        break;
    default:
        facet_kernel<R, MODE, 8><<<blocks, 96, 0, s>>>(m, pst);
        break;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_unkick(const DeviceModel &m, double *out12, cudaStream_t s)
{
    const int64_t n = 6 * (int64_t)m.N;
    if (n == 0) return cudaSuccess;
    unkick_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, out12);
    return cudaGetLastError();
}

cudaError_t launch_kick(const DeviceModel &m, cudaStream_t s)
{
    const int64_t n = 6 * (int64_t)m.N;
    if (n == 0) return cudaSuccess;
    kick_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_facet(const DeviceModel &m, int mode, const void *src_override, cudaStream_t s)
{
    const void *pst = src_override ? src_override
                                   : (sizeof(R) == 4 ? static_cast<const void *>(m.pm32)
                                                     : static_cast<const void *>(m.pstate));
    switch (mode) {
    case FACET_FROM_HIST:
        return launch_facet_tpb<R, FACET_FROM_HIST>(m, pst, s);
    case FACET_ELASTIC:
        return launch_facet_tpb<R, FACET_ELASTIC>(m, pst, s);
    case FACET_METRIC:
        return launch_facet_tpb<R, FACET_METRIC>(m, pst, s);
    default:
        return launch_facet_tpb<R, FACET_STEP>(m, pst, s);
    }
}

template <class R, int LPP>
cudaError_t launch_gather_lpp(const DeviceModel &m, int mode, double *out6, cudaStream_t s)
{
    const int64_t warps = ((int64_t)m.N + (32 / LPP) - 1) / (32 / LPP);
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    switch (mode) {
    case GATHER_ASSEMBLE:
        gather_kernel<R, GATHER_ASSEMBLE, LPP><<<blocks, 256, 0, s>>>(m, out6);
        break;
    default:
        gather_kernel<R, GATHER_STEP_MID, LPP><<<blocks, 256, 0, s>>>(m, out6);
        break;
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_gather(const DeviceModel &m, int mode, double *out6, cudaStream_t s)
{
    if (m.N == 0) return cudaSuccess;
    switch (m.gather_lanes) {
    case 32:
        return launch_gather_lpp<R, 32>(m, mode, out6, s);
    case 16:
        return launch_gather_lpp<R, 16>(m, mode, out6, s);
    default:
        return launch_gather_lpp<R, 8>(m, mode, out6, s);
    }
}

cudaError_t launch_mirror(const DeviceModel &m, cudaStream_t s)
{
    if (!m.pm32 || m.N == 0) return cudaSuccess;
    mirror_kernel<<<(unsigned)((m.N + 255) / 256), 256, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_energy(const DeviceModel &m, int32_t p0, int32_t p1, double *partial, double *out16,
                          cudaStream_t s)
{
    const int32_t nb = (p1 - p0 + 255) / 256;
    if (nb <= 0) return cudaMemsetAsync(out16, 0, 16 * sizeof(double), s);
    energy_kernel<<<nb, 256, 0, s>>>(m, p0, p1, partial);
    energy_final_kernel<<<1, 256, 0, s>>>(partial, nb, out16);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_hist_to_user(const DeviceModel &m, double *out5, cudaStream_t s)
{
    const int64_t n = 12 * (int64_t)m.T;
    if (n == 0) return cudaSuccess;
    hist_to_user_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, out5);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_hist_from_user(const DeviceModel &m, const double *in5, cudaStream_t s)
{
    const int64_t n = 12 * (int64_t)m.T;
    if (n == 0) return cudaSuccess;
    hist_from_user_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, in5);
    return cudaGetLastError();
}

template cudaError_t launch_facet<float>(const DeviceModel &, int, const void *, cudaStream_t);
template cudaError_t launch_facet<double>(const DeviceModel &, int, const void *, cudaStream_t);
template cudaError_t launch_gather<float>(const DeviceModel &, int, double *, cudaStream_t);
template cudaError_t launch_gather<double>(const DeviceModel &, int, double *, cudaStream_t);
template cudaError_t launch_hist_to_user<float>(const DeviceModel &, double *, cudaStream_t);
template cudaError_t launch_hist_to_user<double>(const DeviceModel &, double *, cudaStream_t);
template cudaError_t launch_hist_from_user<float>(const DeviceModel &, const double *, cudaStream_t);
template cudaError_t launch_hist_from_user<double>(const DeviceModel &, const double *, cudaStream_t);

}  // namespace ldpm
