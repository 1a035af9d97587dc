// ldpm_device.cuh -- device helpers shared by the kernel translation units (ldpm_kernels.cu,
// ldpm_adjoint.cu): small vector algebra, the Appendix A facet law, FP64 <-> FP32 conversions on the
// integer pipe, the boundary-condition ramp.  Not part of the public ABI.
#pragma once

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
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }

// Exponentials of the facet law.  Mixed mode: the hardware approximations (exp via ex2, x^y via
// lg2/ex2; errors of a few ulp, far inside the mixed-mode tolerances).  This translation unit is
// compiled with approximate FP32 division and square root (-prec-div=false -prec-sqrt=false), which
// touches only the mixed-mode arithmetic.  FP64 mode: the library exp and log.  The law's only power
// is (2 omega / pi)^n_t with a base in [0, 1] and a small exponent, so exp(n_t log x) is within a few
// ulp of x^n_t.  With it and the library rsqrt in place of pow and 1 / sqrt, the FP64 facet pass
// takes 5 % less time on GB300 (1124 -> 1067 us on 1.82M facets).
__device__ __forceinline__ float exp_(float x) { return __expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }
// x^y for x >= 0, y >= 0
__device__ __forceinline__ float powpos_(float x, float y)
{
    return x > 0.0f ? exp2f(y * __log2f(x)) : (y == 0.0f ? 1.0f : 0.0f);
}
__device__ __forceinline__ double powpos_(double x, double y)
{
    return x > 0.0 ? exp(y * log(x)) : (y == 0.0 ? 1.0 : 0.0);
}

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

// Constants of the law for a facet with its own E0, alpha, sigma_t: the ones that depend on them are
// rebuilt from the material's ratios.
template <class R>
__device__ __forceinline__ LawConst<R> facet_params(const LawConst<R> &c, R E0, R alpha, R sigma_t)
{
    LawConst<R> p = c;
    p.E0 = E0;
    p.alpha = alpha;
    p.inv_alpha = R(1) / alpha;
    p.sigma_t = sigma_t;
    p.four_alpha_over_r2 = alpha * c.four_over_r2;
    p.Hs_over_alpha = c.r_s * E0 * p.inv_alpha;
    p.Hc0 = c.Hc0_E0 * E0;
    p.Hc1 = c.Hc1_E0 * E0;
    p.ec0 = c.sigma_c0 / E0;
    p.ec1 = c.kc0 * p.ec0;
    p.eV0 = c.kc3 * p.ec0;
    p.Ed = c.Ed_E0 * E0;
    p.sigma_s = c.r_st * sigma_t;
    return p;
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
        R d_eff = num / (eeff + e_old);
        const R t_old = sqrt(tN * tN + (tM * tM + tL * tL) * c.inv_alpha);
        if (c.k_t > R(0) && t_old <= R(0) && d_eff > R(0)) {
            // reloading from zero traction: it stays zero up to e_tr = k_t (e_max - sigma_bt / E0)
            const R e_tr = c.k_t * (emax - sigma_bt / E0);
            if (e_tr > e_old) d_eff = eeff > e_tr ? eeff - e_tr : R(0);
        }
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
// Round to nearest, ties to even: the 29 dropped mantissa bits decide whether the kept 23-bit
// mantissa is incremented (a carry out of the mantissa moves to the exponent, up to infinity).
// Outside the normal float range it falls back to d2f_trunc.
__device__ __forceinline__ float d2f_rn(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    if (e <= 0 || e >= 255) return d2f_trunc(x);
    const uint32_t m23 = (uint32_t)((b >> 29) & 0x7fffffu);
    const uint32_t rest = (uint32_t)b & 0x1fffffffu;
    const uint32_t u = ((uint32_t)(b >> 32) & 0x80000000u) | ((uint32_t)e << 23) | m23;
    const bool up = rest > 0x10000000u || (rest == 0x10000000u && (m23 & 1u));
    return __uint_as_float(u + (up ? 1u : 0u));
}

__device__ __forceinline__ double f2d_bits(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0) return __longlong_as_double((long long)sign);
    const uint64_t ed = e == 255 ? 0x7ffull : (uint64_t)(e + 896);
    return __longlong_as_double((long long)(sign | (ed << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
}

// ------------------------------------------------------------------------------------------------
// Compensated ("float-float") arithmetic on the FP32 pipe.  A value is the unevaluated sum hi + lo of
// two floats (48 mantissa bits).  two_sum is Knuth's error-free addition (TAOCP vol. 2, 4.2.2):
// s + e == a + b exactly; fast_two_sum is Dekker's (1971) for |a| >= |b|; the product's rounding
// error is exact with one FMA.  The mixed mode sums forces and energies with these: the GB300 FP64
// pipe issues one warp instruction per ~64 cycles per sub-partition, the FP32 pipe one per cycle.
// Every operation is written with explicit round-to-nearest intrinsics so the compiler neither
// contracts nor reorders them.
// ------------------------------------------------------------------------------------------------
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// a += x (x a float): the rounding error of the running sum is collected in a.lo
__device__ __forceinline__ void ff_acc(ff &a, float x)
{
    const ff t = two_sum(a.hi, x);
    a.hi = t.hi;
    a.lo = __fadd_rn(a.lo, t.lo);
}
// a += x (x a float-float)
__device__ __forceinline__ void ff_acc(ff &a, ff x)
{
    const ff t = two_sum(a.hi, x.hi);
    a.hi = t.hi;
    a.lo = __fadd_rn(a.lo, __fadd_rn(t.lo, x.lo));
}
__device__ __forceinline__ ff ff_norm(ff a) { return fast_two_sum(a.hi, a.lo); }
// a + b; absolute error below ~2^-46 (|a| + |b|), the form of an FP64 addition's bound
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_shfl_xor(ff a, int off)
{
    return {__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off)};
}
// FP64 value as a float-float (integer-pipe split; relative error below 2^-46) and back (one FP64
// addition of two exactly converted floats).
__device__ __forceinline__ ff ff_from_double(double x)
{
    ff r;
    d2f_split(x, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ double ff_to_double(ff a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

// The same arithmetic on two float-float values at once (components x and y), with the packed FP32
// instructions of sm_100 and later (one instruction per pair).  a - b is fma(b, -1, a): the product is
// exact, so the single rounding equals that of a subtraction, and each component is bitwise the
// scalar operation's result.
struct ff2 {
    float2 hi, lo;
};
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ ff2 two_sum2(float2 a, float2 b)
{
    const float2 s = __fadd2_rn(a, b);
    const float2 bb = f2_sub(s, a);
    return {s, __fadd2_rn(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb))};
}
__device__ __forceinline__ ff2 fast_two_sum2(float2 a, float2 b)
{
    const float2 s = __fadd2_rn(a, b);
    return {s, f2_sub(b, f2_sub(s, a))};
}
// a += x, componentwise (x a pair of floats)
__device__ __forceinline__ void ff2_acc(ff2 &a, float2 x)
{
    const ff2 t = two_sum2(a.hi, x);
    a.hi = t.hi;
    a.lo = __fadd2_rn(a.lo, t.lo);
}
__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b)
{
    const ff2 s = two_sum2(a.hi, b.hi);
    return fast_two_sum2(s.hi, __fadd2_rn(s.lo, __fadd2_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff2 ff2_shfl_xor(ff2 a, int off)
{
    ff2 r;
    r.hi.x = __shfl_xor_sync(0xffffffffu, a.hi.x, off);
    r.hi.y = __shfl_xor_sync(0xffffffffu, a.hi.y, off);
    r.lo.x = __shfl_xor_sync(0xffffffffu, a.lo.x, off);
    r.lo.y = __shfl_xor_sync(0xffffffffu, a.lo.y, off);
    return r;
}
__device__ __forceinline__ ff2 ff2_pack(ff x, ff y) { return {make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)}; }

// Sum of three float-float pairs (components 0-1, 2-3, 4-5) over each aligned group of 8 lanes by
// halving exchanges on pairs (the three padded with a zero pair to four: 2 + 1 pair additions, then
// one scalar).  Afterwards lane L (L = lane & 7) holds the group sum of component L for L < 6 and
// zero for L = 6, 7.  The order of the additions is fixed.
__device__ __forceinline__ ff pair_halving_sum6(const ff2 (&v)[3], int lane)
{
    const ff2 zero = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
    ff2 w0, w1;
    {
        const bool upper = (lane & 4) != 0;
        const ff2 keep0 = upper ? v[2] : v[0], give0 = upper ? v[0] : v[2];
        const ff2 keep1 = upper ? zero : v[1], give1 = upper ? v[1] : zero;
        w0 = ff2_add(keep0, ff2_shfl_xor(give0, 4));
        w1 = ff2_add(keep1, ff2_shfl_xor(give1, 4));
    }
    ff2 u;
    {
        const bool upper = (lane & 2) != 0;
        const ff2 keep = upper ? w1 : w0, give = upper ? w0 : w1;
        u = ff2_add(keep, ff2_shfl_xor(give, 2));
    }
    const bool upper = (lane & 1) != 0;
    const ff keep = upper ? ff{u.hi.y, u.lo.y} : ff{u.hi.x, u.lo.x};
    const ff give = upper ? ff{u.hi.x, u.lo.x} : ff{u.hi.y, u.lo.y};
    return ff_add(keep, ff_shfl_xor(give, 1));
}

// Accumulator operations shared by the FP64 sums (double) and the mixed-mode sums (float-float).
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ ff acc_add(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ double acc_shfl_xor(double a, int off) { return __shfl_xor_sync(0xffffffffu, a, off); }
__device__ __forceinline__ ff acc_shfl_xor(ff a, int off) { return ff_shfl_xor(a, off); }

// Sum of v[0..5] over each aligned group of 8 lanes, by halving exchanges: at each level a lane keeps
// half of its values (the upper half when its lane bit is set) and adds its partner's copy of that
// half (3 + 2 + 1 additions instead of 3 x 6; the second level pads its 3 values with a zero).
// Afterwards v[0] of lane L (L = lane & 7) holds the group sum of value kHalvingSlot[L]: lanes
// 0, 1, 2, 4, 5, 6 hold values 0..5, lanes 3 and 7 zero.  The order of the additions is fixed.
template <class A>
__device__ __forceinline__ void halving_sum6(A (&v)[6], int lane)
{
    A w[4];
    {
        const bool upper = (lane & 4) != 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const A keep = upper ? v[3 + i] : v[i];
            const A give = upper ? v[i] : v[3 + i];
            w[i] = acc_add(keep, acc_shfl_xor(give, 4));
        }
        w[3] = A{};
    }
    {
        const bool upper = (lane & 2) != 0;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const A keep = upper ? w[2 + i] : w[i];
            const A give = upper ? w[i] : w[2 + i];
            w[i] = acc_add(keep, acc_shfl_xor(give, 2));
        }
    }
    {
        const bool upper = (lane & 1) != 0;
        const A keep = upper ? w[1] : w[0];
        const A give = upper ? w[0] : w[1];
        v[0] = acc_add(keep, acc_shfl_xor(give, 1));
    }
}
// Component held by lane L of an 8-lane group after halving_sum6 (-1: none).
__device__ __forceinline__ int halving_slot6(int L) { return L < 3 ? L : (L == 3 || L == 7 ? -1 : L - 1); }

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

}  // namespace
}  // namespace ldpm
