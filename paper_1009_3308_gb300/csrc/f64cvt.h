// Conversions between binary64 and binary32 on the integer ALU: binary64 ->
// binary32 rounds to nearest, ties to even (IEEE 754 convertFormat), and
// binary32 -> binary64 is exact.  GB300's FP64 pipe is narrow (a few
// operations per clock per SM), and a conversion instruction goes through
// it: kernels that convert many FP64 inputs use this instead.
//
// A result in the normal binary32 range is formed from the bits directly:
// the 23 leading fraction bits of the binary64 value, the 29 dropped bits
// deciding the rounding (above half: up; exactly half: to the even
// neighbour); a carry out of the fraction raises the exponent, and out of
// the largest finite exponent gives infinity, as the standard requires.
// Zeros are returned directly; results below the normal range (binary32
// subnormals) and infinities or NaNs take the compiler's own conversion.
//
// Host and device code (tests compile it on the host and compare it with the
// host's own conversion).
#pragma once
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define SPH_HD __host__ __device__ __forceinline__
#else
#define SPH_HD inline
#endif

namespace sph {

SPH_HD float f64_to_f32_rn(double x) {
    uint64_t b;
#if defined(__CUDA_ARCH__)
    b = static_cast<uint64_t>(__double_as_longlong(x));
#else
    std::memcpy(&b, &x, sizeof b);
#endif
    const uint32_t hi = uint32_t(b >> 32), lo = uint32_t(b);
    const uint32_t sign = hi & 0x80000000u;
    const int e = int((hi >> 20) & 0x7FFu) - 1023 + 127;   // binary32 biased exponent
    uint32_t f;
    if (e >= 1 && e <= 254) {
        const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // 23 fraction bits
        const uint32_t r = lo & 0x1FFFFFFFu;                      // 29 dropped bits
        f = sign | (uint32_t(e) << 23) | m;
        if (r > 0x10000000u || (r == 0x10000000u && (m & 1u))) f += 1u;
    } else if ((hi & 0x7FFFFFFFu) == 0u && lo == 0u) {
        f = sign;   // +-0
    } else {
#if defined(__CUDA_ARCH__)
        return __double2float_rn(x);
#else
        return static_cast<float>(x);
#endif
    }
#if defined(__CUDA_ARCH__)
    return __uint_as_float(f);
#else
    float y;
    std::memcpy(&y, &f, sizeof y);
    return y;
#endif
}

// Binary32 -> binary64, exact, on the integer ALU: the exponent is rebiased
// and the fraction widened.  Zeros are formed directly; binary32 subnormals,
// infinities and NaNs take the compiler's own conversion.
SPH_HD double f32_to_f64(float x) {
    uint32_t u;
#if defined(__CUDA_ARCH__)
    u = __float_as_uint(x);
#else
    std::memcpy(&u, &x, sizeof u);
#endif
    const uint32_t e = (u >> 23) & 0xFFu;
    uint64_t b;
    if (e != 0u && e != 0xFFu) {
        b = (uint64_t(u & 0x80000000u) << 32) | (uint64_t(e - 127u + 1023u) << 52) | (uint64_t(u & 0x7FFFFFu) << 29);
    } else if ((u & 0x7FFFFFFFu) == 0u) {
        b = uint64_t(u) << 32;   // +-0
    } else {
        return static_cast<double>(x);
    }
#if defined(__CUDA_ARCH__)
    return __longlong_as_double(static_cast<long long>(b));
#else
    double y;
    std::memcpy(&y, &b, sizeof y);
    return y;
#endif
}

}  // namespace sph

#undef SPH_HD
