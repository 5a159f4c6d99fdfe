// Binary64 -> binary32 conversion, round to nearest, ties to even (IEEE 754
// convertFormat), on the integer ALU.  GB300's FP64 pipe is narrow (a few
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

}  // namespace sph

#undef SPH_HD
