// dt_trig.cuh -- sine and cosine of a roll angle |x| <= pi/2 for the roll search of the
// disparity transformation, with a short FP64 dependency chain.
//
// Both come from their Taylor series about 0:
//     sin x = sum_k (-1)^k x^(2k+1) / (2k+1)!,  k = 0..10  (first omitted term x^23/23! < 1.4e-18)
//     cos x = sum_k (-1)^k x^(2k)   / (2k)!,    k = 0..11  (first omitted term x^24/24! < 1e-19)
// for |x| <= pi/2.  The polynomials in y = x^2 are evaluated by Estrin's scheme (pairs of
// coefficients combined with y, pairs of pairs with y^2, then y^4 and y^8), which needs six
// dependent FP64 operations where Horner's rule needs twelve: on GB300 an FP64 FMA has a
// latency of about 65 cycles, and the search is one dependency chain.  Every step is an
// explicit fma() or product, so host and device builds compute the same values.
#pragma once
#include <math.h>

#if defined(__CUDACC__)
#define SGB_HD __host__ __device__ __forceinline__
#else
#define SGB_HD inline
#endif

namespace sgb {

// (-1)^k / (2k+1)! and (-1)^k / (2k)!, each rounded once from the exact rational
#define SGB_F(n) (1.0 / (n))
constexpr double kSinC[11] = {1.0, -SGB_F(6.0), SGB_F(120.0), -SGB_F(5040.0), SGB_F(362880.0),
                              -SGB_F(39916800.0), SGB_F(6227020800.0), -SGB_F(1307674368000.0),
                              SGB_F(355687428096000.0), -SGB_F(121645100408832000.0),
                              SGB_F(51090942171709440000.0)};
constexpr double kCosC[12] = {1.0, -SGB_F(2.0), SGB_F(24.0), -SGB_F(720.0), SGB_F(40320.0),
                              -SGB_F(3628800.0), SGB_F(479001600.0), -SGB_F(87178291200.0),
                              SGB_F(20922789888000.0), -SGB_F(6402373705728000.0),
                              SGB_F(2432902008176640000.0), -SGB_F(1124000727777607680000.0)};
#undef SGB_F

SGB_HD void sincos_half_pi(double x, double *s, double *c)
{
    const double y = x * x, y2 = y * y, y4 = y2 * y2, y8 = y4 * y4;
    // sin: x * (a0 + a1 y + ... + a10 y^10)
    const double sp0 = fma(kSinC[1], y, kSinC[0]), sp1 = fma(kSinC[3], y, kSinC[2]);
    const double sp2 = fma(kSinC[5], y, kSinC[4]), sp3 = fma(kSinC[7], y, kSinC[6]);
    const double sp4 = fma(kSinC[9], y, kSinC[8]);
    const double sq0 = fma(sp1, y2, sp0), sq1 = fma(sp3, y2, sp2), sq2 = fma(kSinC[10], y2, sp4);
    const double sr0 = fma(sq1, y4, sq0);
    *s = x * fma(sq2, y8, sr0);
    // cos: b0 + b1 y + ... + b11 y^11
    const double cp0 = fma(kCosC[1], y, kCosC[0]), cp1 = fma(kCosC[3], y, kCosC[2]);
    const double cp2 = fma(kCosC[5], y, kCosC[4]), cp3 = fma(kCosC[7], y, kCosC[6]);
    const double cp4 = fma(kCosC[9], y, kCosC[8]), cp5 = fma(kCosC[11], y, kCosC[10]);
    const double cq0 = fma(cp1, y2, cp0), cq1 = fma(cp3, y2, cp2), cq2 = fma(cp5, y2, cp4);
    const double cr0 = fma(cq1, y4, cq0);
    *c = fma(cq2, y8, cr0);
}

}  // namespace sgb
