// row_shift.cuh -- the integer row shift s_i = floor(s + 0.5) of §3.1 in FP32, exact for every
// float s.
//
// s + 0.5 rounded to float can round up to the next integer (s = 0.5 - 2^-25 gives 1.0 where
// the exact value floors to 0), so with f = floor(s) the test is s >= f + 0.5, and f + 0.5 is a
// float for |s| < 2^22.  For 2^22 <= |s| < 2^23, s + 0.5 is exact (the spacing of s is 0.5);
// from 2^23 on, s is an integer.  A NaN comes back as NaN.  (FP64 would also be exact, but an
// FP64 instruction costs a warp about as much as 64 FP32 ones on GB300.)
#pragma once
#include <math.h>

#if defined(__CUDACC__)
#define SGB_RS_HD __host__ __device__ __forceinline__
#else
#define SGB_RS_HD inline
#endif

namespace sgb {

SGB_RS_HD float round_half_up(float s)
{
    const float as = fabsf(s);
    if (as < 4194304.f) {
        const float f = floorf(s);
        return s >= f + 0.5f ? f + 1.f : f;
    }
    return as < 8388608.f ? floorf(s + 0.5f) : s;
}

}  // namespace sgb
