// Double-precision arithmetic helpers shared by the K1 kernels and the
// measurement probes (probe.cu tests them against CUDA's own division).
#pragma once

#include <cuda_runtime.h>

namespace ptp {

// 1/d for d in [2^-126, 2^127] (the normal float range) by the Newton-Raphson
// iteration for the reciprocal, x <- x (2 - d x) = x + x (1 - d x), started
// from the single-precision reciprocal of d rounded to float (relative error
// below 2^-23).  The relative error squares at every step (2^-46, then below
// the double rounding), so two steps reach double precision: the result is
// within a few units in the last place of the correctly rounded 1/d.
__device__ __forceinline__ double recip_newton(double d) {
    double x = (double)__frcp_rn(__double2float_rn(d));
    double e = fma(-d, x, 1.0);
    x = fma(x, e, x);
    e = fma(-d, x, 1.0);
    return fma(x, e, x);
}

}  // namespace ptp
