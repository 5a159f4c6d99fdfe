// Complex arithmetic and small in-register DFTs (radix 2, 3, 4, 8) shared by
// the longitude ("ring") transforms: y_r = sum_s v_s e^{sign 2 pi i r s / R}.
#pragma once
#include <cuda_runtime.h>

namespace sph {

template <typename T> struct cx { T x, y; };

template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

template <typename T, typename TW>
__device__ __forceinline__ cx<T> twiddle(const TW* tw, int t, int sign) {
    // tw holds e^{-2 pi i t / M}; the inverse transform (sign = +1) uses its conjugate
    cx<T> w{T(tw[2 * t]), T(tw[2 * t + 1])};
    if (sign > 0) w.y = -w.y;
    return w;
}

// small DFTs: y_r = sum_s v_s e^{sign 2 pi i r s / R}
template <typename T>
__device__ __forceinline__ void dft2(cx<T>* v) {
    cx<T> a = v[0], b = v[1];
    v[0] = {a.x + b.x, a.y + b.y};
    v[1] = {a.x - b.x, a.y - b.y};
}
template <typename T>
__device__ __forceinline__ void dft3(cx<T>* v, int sign) {
    const T h = T(0.86602540378443864676);  // sqrt(3)/2
    cx<T> t1{v[1].x + v[2].x, v[1].y + v[2].y};
    cx<T> t2{v[0].x - T(0.5) * t1.x, v[0].y - T(0.5) * t1.y};
    cx<T> t3{T(sign) * h * (v[1].x - v[2].x), T(sign) * h * (v[1].y - v[2].y)};
    v[0] = {v[0].x + t1.x, v[0].y + t1.y};
    v[1] = {t2.x - t3.y, t2.y + t3.x};  // t2 + i t3
    v[2] = {t2.x + t3.y, t2.y - t3.x};  // t2 - i t3
}
template <typename T>
__device__ __forceinline__ void dft4(cx<T>* v, int sign) {
    cx<T> a0{v[0].x + v[2].x, v[0].y + v[2].y};
    cx<T> a1{v[0].x - v[2].x, v[0].y - v[2].y};
    cx<T> b0{v[1].x + v[3].x, v[1].y + v[3].y};
    cx<T> b1{v[1].x - v[3].x, v[1].y - v[3].y};
    // (sign i) * b1
    cx<T> ib1{-T(sign) * b1.y, T(sign) * b1.x};
    v[0] = {a0.x + b0.x, a0.y + b0.y};
    v[2] = {a0.x - b0.x, a0.y - b0.y};
    v[1] = {a1.x + ib1.x, a1.y + ib1.y};
    v[3] = {a1.x - ib1.x, a1.y - ib1.y};
}

// radix 8 = two radix-4 DFTs of the even/odd samples and a radix-2 combine
// with the eighth roots of unity w^r = e^{sign 2 pi i r / 8}
template <typename T>
__device__ __forceinline__ void dft8(cx<T>* v, int sign) {
    cx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cx<T> o[4] = {v[1], v[3], v[5], v[7]};
    dft4(e, sign);
    dft4(o, sign);
    const T h = T(0.70710678118654752440);  // sqrt(2)/2
    const T sg = T(sign);
    // w^1 = h (1, sign), w^2 = (0, sign), w^3 = h (-1, sign)
    cx<T> t1{h * (o[1].x - sg * o[1].y), h * (o[1].y + sg * o[1].x)};
    cx<T> t2{-sg * o[2].y, sg * o[2].x};
    cx<T> t3{h * (-o[3].x - sg * o[3].y), h * (-o[3].y + sg * o[3].x)};
    v[0] = {e[0].x + o[0].x, e[0].y + o[0].y};
    v[4] = {e[0].x - o[0].x, e[0].y - o[0].y};
    v[1] = {e[1].x + t1.x, e[1].y + t1.y};
    v[5] = {e[1].x - t1.x, e[1].y - t1.y};
    v[2] = {e[2].x + t2.x, e[2].y + t2.y};
    v[6] = {e[2].x - t2.x, e[2].y - t2.y};
    v[3] = {e[3].x + t3.x, e[3].y + t3.y};
    v[7] = {e[3].x - t3.x, e[3].y - t3.y};
}

template <typename T, int R>
__device__ __forceinline__ void dft(cx<T>* v, int sign) {
    if constexpr (R == 8) dft8(v, sign);
    else if constexpr (R == 4) dft4(v, sign);
    else if constexpr (R == 2) dft2(v);
    else dft3(v, sign);
}

}  // namespace sph
