// Segment weights of the linear-in-tau source integral, FP64 and FP32 forms,
// shared by the formal-solution kernels (device code only).
//
// Over a segment of optical depth x the intensity gains
//   w_cur S(downstream) + w_up S(upstream),
//   w_cur = 1 - (1-e)/x,  w_up = (1-e)/x - e,  e = exp(-x),
// the exact integral of S(t) e^{-t} for S linear in t.  With
// phi2(z) = (e^z - 1 - z)/z^2 = sum_{n>=0} z^n/(n+2)!  these are
//   w_cur = x phi2(-x),  w_up = e x phi2(x),  e = 1 - x + x w_cur,
// and phi2(+-x) = E +- O with E = sum_j x^{2j}/(2j+2)!,
// O = x sum_j x^{2j}/(2j+3)!: a cancellation-free form for small x.
#pragma once

#include <cuda_runtime.h>

namespace rt3d {
namespace {

// ---- FP64 -----------------------------------------------------------------
//
// The FP64 pipe of GB300 issues about 2 DFMA per SM per clock, so the FP64
// weights are written to use few FP64 instructions:
//
//  x < 1/4: the phi2 series (Horner in z = x^2, six terms each: the first
//    omitted terms, z^6/14! and z^6/15! at z <= 1/16, are below 7e-19 and
//    5e-20); no exp call and no cancellation.  With E as above and
//    O = x Q, w_cur = xE - zQ and w_up = e (xE + zQ): 17 FP64 operations.
//  x >= 1/4: e from Tang's table-driven method (ACM TOMS 15, 1989):
//    -x/ln2 = k/256 + r/ln2, k = round(-256 x/ln2), |r| <= ln2/512,
//    e = 2^{k>>8} * 2^{(k&255)/256} * P(r), P the degree-4 Taylor polynomial
//    of e^r (relative error < 4e-17), the 256 powers 2^{j/256} in shared
//    memory; then (1-e)/x from a reciprocal seed and two Newton steps.
//    Above x = 700 e is taken as 0 (it would scale I by < 1e-304).
//  Both branch tests compare the high word of x (x >= 0) as an integer, so
//    they take no FP64 compare.

constexpr int kExpTable = 256;

// Fill tab[j] = 2^{j/256} (call from every thread, then __syncthreads()).
__device__ __forceinline__ void fill_exp_table(double* tab)
{
    for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) tab[j] = exp2((double)j / kExpTable);
}

__device__ __forceinline__ double exp_neg_tang(double x, const double* __restrict__ tab)
{
    constexpr double kMagic = 6755399441055744.0;          // 1.5 * 2^52: round to integer
    constexpr double kInvL = 369.329930467574632284140718;  // 256 / ln 2
    constexpr double kL1 = 2.7076061740622863e-03;          // ln2/256, leading part
    constexpr double kL2 = 9.058776616587108e-20;           // ln2/256 - kL1
    const double t = fma(-x, kInvL, kMagic);
    const int k = __double2loint(t);                         // round(-256 x / ln2)
    const double kd = t - kMagic;
    double r = fma(-kd, kL1, -x);
    r = fma(-kd, kL2, r);
    double p = fma(fma(fma(1.0 / 24.0, r, 1.0 / 6.0), r, 0.5), r, 1.0);
    p = fma(p, r, 1.0);
    const double e = tab[k & (kExpTable - 1)] * p;
    // scale by 2^(k >> 8): add to the exponent field (result stays normal for x <= 700)
    return __hiloint2double(__double2hiint(e) + (k >> 8) * (1 << 20), __double2loint(e));
}

__device__ __forceinline__ double recip_newton(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

constexpr int kHiQuarter = 0x3FD00000;   // high word of 0.25
constexpr int kHi700 = 0x4085E000;       // high word of 700.0

__device__ __forceinline__ void seg_weights64(double x, const double* __restrict__ tab, double& wc,
                                              double& wu, double& e)
{
    const int hx = __double2hiint(x);
    if (hx < kHiQuarter) {
        const double z = x * x;
        // E = sum_j z^j/(2j+2)!,  Q = sum_j z^j/(2j+3)!  (j = 0..5)
        double E = fma(fma(fma(fma(1.0 / 479001600.0, z, 1.0 / 3628800.0), z, 1.0 / 40320.0), z,
                           1.0 / 720.0), z, 1.0 / 24.0);
        E = fma(E, z, 0.5);
        double Q = fma(fma(fma(fma(1.0 / 6227020800.0, z, 1.0 / 39916800.0), z, 1.0 / 362880.0), z,
                           1.0 / 5040.0), z, 1.0 / 120.0);
        Q = fma(Q, z, 1.0 / 6.0);
        const double xE = x * E;
        wc = fma(-z, Q, xE);
        e = fma(x, wc, 1.0 - x);
        wu = e * fma(z, Q, xE);
    } else {
        e = hx < kHi700 ? exp_neg_tang(x, tab) : 0.0;
        const double q = (1.0 - e) * recip_newton(x);
        wc = 1.0 - q;
        wu = q - e;
    }
}

// Cutoff test on exponent fields only (integer pipe).  With T < 2^(eT+1),
// smax < 2^(es+1), |I| >= 2^eI and cut >= 2^-lc (lc = ceil(-log2 cut)),
// eI - eT >= es + lc + 2 guarantees T * smax <= cut * |I|, i.e. the rest of
// the characteristic changes I by at most cut * |I|.  `need` = es + lc + 2.
__device__ __forceinline__ bool cut_now(double T, double I, int need)
{
    const int eT = (__double2hiint(T) >> 20) & 0x7ff;
    const int eI = (__double2hiint(I) >> 20) & 0x7ff;
    return eI - eT >= need;
}

__device__ __forceinline__ int cut_need(double smax, double cut)
{
    // cut <= 0 disables the test (need larger than any exponent gap)
    if (!(cut > 0.0)) return 4096;       // never cut
    if (!(smax > 0.0)) return -4096;     // S = 0 and no boundary intensity: I = 0 exactly
    const int es = ((__double2hiint(smax) >> 20) & 0x7ff) - 1023;
    const int lc = (int)ceil(-log2(cut));
    return es + lc + 2;
}

// ---- FP32 -----------------------------------------------------------------
//
//  x < 2: phi2(+-x) = E(z) +- x Q(z) with E, Q degree-4 polynomials in
//  z = x^2 fitted on z in [0, 4] for the least maximum relative error
//  (fit_weights32.py: 1.9e-8 for E, 3.0e-8 for Q with the coefficients
//  rounded to FP32, against 2e-9 truncation for seven Taylor terms each);
//  x >= 2: closed form (1-e loses nothing there).  e from the MUFU ex2.
__device__ __forceinline__ float ex2_approx(float y)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}

__device__ __forceinline__ float rcp_approx(float y)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}

// E(z) and Q(z), z = x^2 < 4: phi2(+-x) = E +- x Q
__device__ __forceinline__ void phi2_eq32(float z, float& E, float& Q)
{
    E = fmaf(fmaf(fmaf(2.968770900e-07f, z, 2.472764936e-05f), z, 1.388992299e-03f), z,
             4.166661575e-02f);
    E = fmaf(E, z, 0.5f);
    Q = fmaf(fmaf(fmaf(2.669341548e-08f, z, 2.749998430e-06f), z, 1.984207920e-04f), z,
             8.333329111e-03f);
    Q = fmaf(Q, z, 1.666666716e-01f);
}

// E = phi2 even part, O = odd part at x < 2 (phi2(+-x) = E +- O)
__device__ __forceinline__ void phi2_parts32(float x, float& E, float& O)
{
    float Q;
    phi2_eq32(x * x, E, Q);
    O = Q * x;
}

__device__ __forceinline__ void seg_weights32(float x, float& wc, float& wu, float& e)
{
    constexpr float kLog2e = 1.4426950408889634f;
    e = ex2_approx(-x * kLog2e);
    if (x < 2.0f) {
        float E, O;
        phi2_parts32(x, E, O);
        wc = x * (E - O);
        wu = (x * e) * (E + O);
    } else {
        const float q = (1.0f - e) * rcp_approx(x);
        wc = 1.0f - q;
        wu = q - e;
    }
}

}  // namespace
}  // namespace rt3d
