// FP64 reciprocals without the FP64 divide.  This part's FP64 units are few
// (about 1/64 of its FP32 rate), and a correctly rounded FP64 division costs
// tens of FP64 instructions; the step controller's kernels would spend most
// of their time in divisions.  Here the FP32 reciprocal (the __frcp_rn
// intrinsic, correctly rounded to 24 bits) seeds Newton-Raphson iterations
// for f(x) = 1/x - d, x <- x + x (1 - d x), each of which squares the
// relative error: one step gives ~2^-47, two give the FP64 rounding level.
// Outside the FP32 normal range the division is used as is.
#pragma once

namespace sph {

template <int STEPS>
__device__ __forceinline__ double rcp64(double d) {
    const double ad = fabs(d);
    if (!(ad > 1.0e-36 && ad < 1.0e36)) return 1.0 / d;
    double x = double(__frcp_rn(float(d)));
#pragma unroll
    for (int s = 0; s < STEPS; ++s) x = fma(x, fma(-d, x, 1.0), x);
    return x;
}

}  // namespace sph
