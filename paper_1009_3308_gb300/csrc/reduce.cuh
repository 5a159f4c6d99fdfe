// Block-wide max-norm reductions for the step controller's weighted norms.
//
// The norms are maxima of non-negative doubles, kept as their bit patterns in
// unsigned 64-bit slots (non-negative IEEE doubles order like their bits), so
// the cross-block combine is one atomicMax per slot and block.  Reducing in
// the block first matters: one atomic per element on a single address
// serialises in L2 (131k same-address atomics per norm at L = 511).
#pragma once
#include <cstdint>

namespace sph {

// slots[idx[j]] = max(slots[idx[j]], max over the block of v[j]) for j < NV.
// Every thread of the block must call it (threads without an element pass 0);
// blockDim.x is a multiple of 32 and at most 1024.  A non-finite value sets
// slots[7] = 1 instead of entering the maximum.
template <int NV>
__device__ __forceinline__ void block_amax(unsigned long long* slots, const double (&v)[NV], const int (&idx)[NV]) {
    __shared__ double red[NV][32];
    double x[NV];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        x[j] = v[j];
        if (!(x[j] <= 1.0e300)) {
            bad = true;
            x[j] = 0.0;
        }
    }
    if (bad) atomicMax(slots + 7, 1ull);
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x[j] = fmax(x[j], __shfl_xor_sync(0xffffffffu, x[j], o));
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) red[j][warp] = x[j];
    __syncthreads();
    if (threadIdx.x < NV) {
        const int j = threadIdx.x;
        double mx = red[j][0];
        for (int w = 1; w < nw; ++w) mx = fmax(mx, red[j][w]);
        if (mx > 0.0) atomicMax(slots + idx[j], static_cast<unsigned long long>(__double_as_longlong(mx)));
    }
}

// FP32 form: the block maximum of NV non-negative floats into the slots
// (converted to double once per block); bad (any thread) sets slots[7].
template <int NV>
__device__ __forceinline__ void block_amax_f(unsigned long long* slots, const float (&v)[NV], const int (&idx)[NV],
                                             bool bad) {
    __shared__ float redf[NV][32];
    float x[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        x[j] = v[j];
        if (!(x[j] <= 3.0e38f)) {
            bad = true;
            x[j] = 0.f;
        }
    }
    if (bad) atomicMax(slots + 7, 1ull);
#pragma unroll
    for (int j = 0; j < NV; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x[j] = fmaxf(x[j], __shfl_xor_sync(0xffffffffu, x[j], o));
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) redf[j][warp] = x[j];
    __syncthreads();
    if (threadIdx.x < NV) {
        const int j = threadIdx.x;
        float mx = redf[j][0];
        for (int w = 1; w < nw; ++w) mx = fmaxf(mx, redf[j][w]);
        if (mx > 0.f) atomicMax(slots + idx[j], static_cast<unsigned long long>(__double_as_longlong(double(mx))));
    }
}

}  // namespace sph
