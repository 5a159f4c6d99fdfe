// Four-step FP32 longitude transform of the RHS for M = 24 M2 (M2 = 4 .. 64)
// as a device function over 128 threads.  It reads the synthesis output
// (order-major or latitude-pair-major) and writes the order-major spectra of
// the analysis directly, without transposes.
//
// With n = t + M2 n1 and k = k1 + 24 k2 (t, k2 < M2; n1, k1 < 24), and
// t = b + B a', k2 = c + A d (M2 = A B):
//   pass 1  (thread t):       24-point DFT over n1, twiddle e^{s 2 pi i t k1 / M}
//   pass 2a (task (k1, b)):   A-point DFT over a', twiddle e^{s 2 pi i b c / M2}
//   pass 2b (task (k1, c)):   B-point DFT over b -> X[k1 + 24 (c + A d)]
// Every thread keeps 24 complex values per signal in registers; the passes
// exchange through padded shared-memory tiles whose strides make every warp
// access conflict-free (B > 1: M2 = 64, 16; one 2-way pass at M2 = 32).
// The pointwise product is taken in the registers of pass 2b, and the forward
// transform of W runs the same factorisation backwards (DFT matrices are
// symmetric): B-point DFT over d, A-point DFT over c, 24-point DFT over k1,
// which leaves W's spectrum in natural order across the threads of pass 1.
// 128 threads hold G = 128 / M2 consecutive rings, so every order-major
// access moves G consecutive latitudes (>= 16 bytes).
#pragma once
#include <cuda_runtime.h>

#include "fft_small.cuh"
#include "internal.h"

namespace sph {

// Padded strides of the shared-memory tiles (found with a bank model of the
// 64-bit accesses of every pass) and the ring buffer length.  SW: pass 2b
// maps thread t to (c, kq2) = (t / B, t % B) instead of (t % A, t / A);
// at M2 = 32 that keeps the one two-way conflicted pass of the unpadded
// element stride in 864 instead of 960 entries, so four CTAs fit an SM.
template <int M2> struct R4;
template <> struct R4<64> { static constexpr int A = 8, P1 = 72, Bp = 9, Q = 72, RING = 1728; static constexpr bool SW = false; };
template <> struct R4<32> { static constexpr int A = 8, P1 = 36, Bp = 4, Q = 35, RING = 864; static constexpr bool SW = true; };
template <> struct R4<16> { static constexpr int A = 4, P1 = 20, Bp = 5, Q = 20, RING = 480; static constexpr bool SW = false; };
template <> struct R4<8> { static constexpr int A = 8, P1 = 9, Bp = 1, Q = 9, RING = 216; static constexpr bool SW = false; };
template <> struct R4<4> { static constexpr int A = 4, P1 = 5, Bp = 1, Q = 5, RING = 124; static constexpr bool SW = false; };

// cos, sin of 2 pi j / 24, j = 0..14
__device__ constexpr double kC24[15] = {1.0, 0.96592582628906828675, 0.86602540378443864676, 0.7071067811865475244,
                                        0.5, 0.25881904510252076235, 0.0, -0.25881904510252076235, -0.5,
                                        -0.7071067811865475244, -0.86602540378443864676, -0.96592582628906828675,
                                        -1.0, -0.96592582628906828675, -0.86602540378443864676};
__device__ constexpr double kS24[15] = {0.0, 0.25881904510252076235, 0.5, 0.7071067811865475244,
                                        0.86602540378443864676, 0.96592582628906828675, 1.0, 0.96592582628906828675,
                                        0.86602540378443864676, 0.7071067811865475244, 0.5, 0.25881904510252076235,
                                        0.0, -0.25881904510252076235, -0.5};

// 24-point DFT in registers, natural order in and out: n = 3 n1 + n2,
// k = k1 + 8 k2 (three 8-point DFTs, twiddles e^{s 2 pi i n2 k1 / 24}, eight
// 3-point DFTs)
template <int S, typename T>
__device__ __forceinline__ void dft24(cx<T>* x) {
    cx<T> u[3][8];
#pragma unroll
    for (int n2 = 0; n2 < 3; ++n2) {
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) u[n2][n1] = x[3 * n1 + n2];
        dft8(u[n2], S);
    }
#pragma unroll
    for (int n2 = 1; n2 < 3; ++n2)
#pragma unroll
        for (int k1 = 1; k1 < 8; ++k1) {
            const int j = n2 * k1;
            u[n2][k1] = cmul(u[n2][k1], cx<T>{T(kC24[j]), T(S * kS24[j])});
        }
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
        cx<T> v[3] = {u[0][k1], u[1][k1], u[2][k1]};
        dft3(v, S);
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) x[k1 + 8 * k2] = v[k2];
    }
}

template <int R, typename T>
__device__ __forceinline__ void dftn(cx<T>* v, int sign) {
    if constexpr (R > 1) dft<T, R>(v, sign);
}

__device__ __forceinline__ cx<float> ld2(const float2* p) {
    const float2 v = *p;
    return {v.x, v.y};
}
__device__ __forceinline__ void st2(float2* p, cx<float> v) { *p = make_float2(v.x, v.y); }
__device__ __forceinline__ cx<float> conjf2(float2 v) { return {v.x, -v.y}; }

struct Ring4Args {
    int N, nlat;
    float two_omega;
    const double* x;       // cos(theta)
    const double* rw;      // (2 pi / M) w_p / sin(theta_p)
    const float2* gsyn;    // three complex spectra, layout gsyn_index(pairs, ...)
    float2* gana;          // [2][N+1][nlat] complex (order-major)
    const float2* ftw;     // tw1 [24][P1] = e^{+2 pi i t k1 / M}, then tw2 [A][B+1] = e^{+2 pi i b c / M2}
    size_t sgs, sga;       // per-instance strides (complex entries) along gridDim.y
    int pairs;             // input layout: latitude-pair-major (1) or order-major (0)
};

// shared memory of one group of G rings: the two signal buffers of every
// ring (the twiddles are read through the L1 cache: every CTA uses the same
// 14 KB)
template <int M2>
__host__ __device__ constexpr size_t ring4_smem() {
    return size_t(2) * (128 / M2) * R4<M2>::RING * sizeof(float2);
}

__device__ __forceinline__ cx<float> ldg2(const float2* p) {
    const float2 v = __ldg(p);
    return {v.x, v.y};
}
__device__ __forceinline__ cx<float> conjg2(const float2* p) {
    const float2 v = __ldg(p);
    return {v.x, -v.y};
}

// The RHS ring transform of the G latitudes lat0 .. lat0 + G - 1 of instance
// inst by 128 threads (tid = 0..127).  sm: ring4_smem<M2>() bytes; s_rw: G
// floats of shared memory; sync(): a barrier over exactly these 128 threads.
// The first barrier comes after the spectra are loaded into registers, so
// consecutive calls may reuse sm.
template <int M2, typename Sync>
__device__ __forceinline__ void ring4_rings(const Ring4Args& a, int lat0, int inst, int tid, float2* sm, float* s_rw,
                                            Sync sync) {
    using C = R4<M2>;
    constexpr int M = 24 * M2, A = C::A, B = M2 / A, P1 = C::P1, Bp = C::Bp, Q = C::Q, RING = C::RING;
    constexpr int G = 128 / M2, GP = G / 2, B2 = B + 1;
    constexpr int TA = 24 / A, TB = 24 / B;
    const float2* __restrict__ tw1 = a.ftw;
    const float2* __restrict__ tw2 = tw1 + 24 * P1;
    float2* buf = sm;
    const int N = a.N, nlat = a.nlat, ld = N + 1;
    const float2* gs = a.gsyn + size_t(inst) * a.sgs;
    float2* ga = a.gana + size_t(inst) * a.sga;

    // stage the spectra: ring r, field f, order m -> buf[r RING + f (N+1) + m].
    // In the latitude-pair-major input, [f][row / 2][m][row % 2], the CTA's
    // pairs are contiguous runs of (N+1) float4 per field; the order-major
    // input gives one float4 per (f, m).  3 (N+1) G / 2 <= 1536 float4 loads
    // per CTA, all of a thread's issued before its stores.
    constexpr int NLD = (3 * 8 * M2 * GP + 127) / 128;
    // element i = tid + 128 k is (order m, pair-field fr) with i = fr ld + m;
    // ld = N + 1 is a runtime value, so (m, fr) advance by steps of 128
    // instead of dividing
    int m0 = tid, fr0 = 0;
    while (m0 >= ld) {
        m0 -= ld;
        ++fr0;
    }
    float4 stv[NLD];
    {
        int m = m0, fr = fr0;
#pragma unroll
        for (int k = 0; k < NLD; ++k) {
            const int rp = fr % GP, f = fr / GP;
            const int pr = lat0 / 2 + rp;
            stv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (f < 3 && 2 * pr < nlat)
                stv[k] = __ldcg(reinterpret_cast<const float4*>(gs + gsyn_index(a.pairs, f, m, 2 * pr, N, nlat)));
            m += 128;
            while (m >= ld) {
                m -= ld;
                ++fr;
            }
        }
    }
    // the previous call's readers of buf and s_rw are done
    sync();
    const int r = tid / M2, t = tid % M2;
    const int lat = lat0 + r;
    const float fc = lat < nlat ? a.two_omega * float(a.x[lat]) : 0.f;
    if (tid < G) s_rw[tid] = lat0 + tid < nlat ? float(a.rw[lat0 + tid]) : 0.f;
    {
        int m = m0, fr = fr0;
#pragma unroll
        for (int k = 0; k < NLD; ++k) {
            const int rp = fr % GP, f = fr / GP;
            if (f < 3) {
                buf[(2 * rp) * RING + f * ld + m] = make_float2(stv[k].x, stv[k].y);
                buf[(2 * rp + 1) * RING + f * ld + m] = make_float2(stv[k].z, stv[k].w);
            }
            m += 128;
            while (m >= ld) {
                m -= ld;
                ++fr;
            }
        }
    }
    sync();
    float2* XA = buf + r * RING;
    float2* XB = buf + (G + r) * RING;

    // pass 1: Hermitian spectra packed as A = zeta + i u_theta, B = u_phi.
    // With M >= 3N + 2, n = t + M2 n1 lies in (N, M - N) for n1 = 8 .. 15, so
    // those inputs are zero for every thread (compile-time, folded into dft24)
    cx<float> xa[24], xb[24];
#pragma unroll
    for (int n1 = 0; n1 < 24; ++n1) {
        const int n = t + M2 * n1;
        cx<float> za{0.f, 0.f}, zb{0.f, 0.f};
        if (n1 >= 8 && n1 < 16) {
        } else if (n <= N) {
            float2 g0 = XA[n], g1 = XA[ld + n], g2 = XA[2 * ld + n];
            if (n == 0) g0.y = g1.y = g2.y = 0.f;
            za = {g0.x - g1.y, g0.y + g1.x};
            zb = {g2.x, g2.y};
        } else if (n >= M - N) {
            const int mm = M - n;
            const float2 g0 = XA[mm], g1 = XA[ld + mm], g2 = XA[2 * ld + mm];
            za = {g0.x + g1.y, g1.x - g0.y};
            zb = {g2.x, -g2.y};
        }
        xa[n1] = za;
        xb[n1] = zb;
    }
    dft24<+1>(xa);
    dft24<+1>(xb);
#pragma unroll
    for (int k1 = 1; k1 < 24; ++k1) {
        const cx<float> w = ldg2(&tw1[k1 * P1 + t]);
        xa[k1] = cmul(xa[k1], w);
        xb[k1] = cmul(xb[k1], w);
    }
    sync();
#pragma unroll
    for (int k1 = 0; k1 < 24; ++k1) {
        st2(&XA[k1 * P1 + t], xa[k1]);
        st2(&XB[k1 * P1 + t], xb[k1]);
    }
    sync();

    // pass 2a: task (k1 = j A + kq, b)
    const int b = t % B, kq = t / B;
    cx<float> ua[TA][A], ub[TA][A];
#pragma unroll
    for (int j = 0; j < TA; ++j) {
        const int k1 = j * A + kq;
#pragma unroll
        for (int ap = 0; ap < A; ++ap) {
            ua[j][ap] = ld2(&XA[k1 * P1 + b + B * ap]);
            ub[j][ap] = ld2(&XB[k1 * P1 + b + B * ap]);
        }
        dftn<A>(ua[j], +1);
        dftn<A>(ub[j], +1);
        if constexpr (B > 1) {
#pragma unroll
            for (int c = 1; c < A; ++c) {
                const cx<float> w = ldg2(&tw2[c * B2 + b]);
                ua[j][c] = cmul(ua[j][c], w);
                ub[j][c] = cmul(ub[j][c], w);
            }
        }
    }
    auto product = [&](cx<float>& za, const cx<float>& zb) {
        // zeta = Re A, u_theta = Im A, u_phi = Re B;  W = (-q u_phi, q u_theta)
        const float q = za.x + fc;
        za = {-q * zb.x, q * za.y};
    };

    // From pass 2b on, the B buffers are free once the B values are in
    // registers: the remaining passes alternate between XA and XB, so each
    // needs one barrier.
    if constexpr (B > 1) {
        sync();
#pragma unroll
        for (int j = 0; j < TA; ++j) {
            const int k1 = j * A + kq;
#pragma unroll
            for (int c = 0; c < A; ++c) {
                st2(&XA[k1 * Q + c * Bp + b], ua[j][c]);
                st2(&XB[k1 * Q + c * Bp + b], ub[j][c]);
            }
        }
        sync();
        // pass 2b: task (k1 = j B + kq2, c) -> X[k1 + 24 (c + A d)]; every
        // task stores W back where it read A
        const int c = C::SW ? t / B : t % A, kq2 = C::SW ? t % B : t / A;
#pragma unroll
        for (int j = 0; j < TB; ++j) {
            const int k1 = j * B + kq2;
            cx<float> va[B], vb[B];
#pragma unroll
            for (int bb = 0; bb < B; ++bb) {
                va[bb] = ld2(&XA[k1 * Q + c * Bp + bb]);
                vb[bb] = ld2(&XB[k1 * Q + c * Bp + bb]);
            }
            dftn<B>(va, +1);
            dftn<B>(vb, +1);
#pragma unroll
            for (int d = 0; d < B; ++d) product(va[d], vb[d]);
            // forward, backwards through the factorisation: B-point DFT over d
            dftn<B>(va, -1);
#pragma unroll
            for (int bb = 1; bb < B; ++bb) va[bb] = cmul(va[bb], conjg2(&tw2[c * B2 + bb]));
#pragma unroll
            for (int bb = 0; bb < B; ++bb) st2(&XA[k1 * Q + c * Bp + bb], va[bb]);
        }
        sync();
        // A-point DFT over c -> a', twiddle e^{-2 pi i t k1 / M} with t = b + B a'
#pragma unroll
        for (int j = 0; j < TA; ++j) {
            const int k1 = j * A + kq;
            cx<float> y[A];
#pragma unroll
            for (int cc = 0; cc < A; ++cc) y[cc] = ld2(&XA[k1 * Q + cc * Bp + b]);
            dftn<A>(y, -1);
#pragma unroll
            for (int ap = 0; ap < A; ++ap) st2(&XB[k1 * P1 + b + B * ap], cmul(y[ap], conjg2(&tw1[k1 * P1 + b + B * ap])));
        }
    } else {
#pragma unroll
        for (int j = 0; j < TA; ++j) {
            const int k1 = j * A + kq;
#pragma unroll
            for (int cc = 0; cc < A; ++cc) product(ua[j][cc], ub[j][cc]);
            dftn<A>(ua[j], -1);
#pragma unroll
            for (int ap = 0; ap < A; ++ap) ua[j][ap] = cmul(ua[j][ap], conjg2(&tw1[k1 * P1 + b + B * ap]));
        }
        sync();
#pragma unroll
        for (int j = 0; j < TA; ++j) {
            const int k1 = j * A + kq;
#pragma unroll
            for (int ap = 0; ap < A; ++ap) st2(&XB[k1 * P1 + b + B * ap], ua[j][ap]);
        }
    }
    sync();
    // 24-point DFT over k1 -> W's spectrum at n = t + M2 n1; only m <= N and
    // m >= M - N are read back: n1 = 8 .. 15 are never needed
    {
        cx<float> y[24];
#pragma unroll
        for (int k1 = 0; k1 < 24; ++k1) y[k1] = ld2(&XB[k1 * P1 + t]);
        dft24<-1>(y);
#pragma unroll
        for (int n1 = 0; n1 < 24; ++n1)
            if (n1 < 8 || n1 >= 16) st2(&XA[t + M2 * n1], y[n1]);
    }
    sync();

    // separate the two real fields, truncate to m <= N, weight, store
    for (int i = tid; i < ld * GP; i += 128) {
        const int rp = i % GP, m = i / GP;
        const int l = lat0 + 2 * rp;
        if (l >= nlat) continue;
        float4 oA, oB;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float2* Z = buf + (2 * rp + e) * RING;
            const float2 p = Z[m], q = Z[(M - m) % M];
            const float sc = s_rw[2 * rp + e];
            const float ax = 0.5f * (p.x + q.x) * sc, ay = 0.5f * (p.y - q.y) * sc;
            const float bx = 0.5f * (p.y + q.y) * sc, by = 0.5f * (q.x - p.x) * sc;
            if (e == 0) {
                oA.x = ax; oA.y = ay; oB.x = bx; oB.y = by;
            } else {
                oA.z = ax; oA.w = ay; oB.z = bx; oB.w = by;
            }
        }
        *reinterpret_cast<float4*>(ga + size_t(m) * nlat + l) = oA;
        *reinterpret_cast<float4*>(ga + size_t(ld + m) * nlat + l) = oB;
    }
}


// The same transform of G = 128 / M2 rings by 256 threads (B > 1, i.e.
// M2 >= 16), for grids too small to fill the GPU: thread tid = 128 h + M2 r
// + t carries one signal of ring r through the inverse passes, A (h = 0) or
// B (h = 1), so each thread's chain holds one 24-point and three A- and
// three B-point DFTs fewer.  In pass 2b the B threads leave their values in
// place in shared memory for the A threads, which take the product and the
// forward transform alone.  Every signal sees the same operations in the
// same order as in ring4_rings, so the results are identical.
template <int M2, typename Sync>
__device__ __forceinline__ void ring4w_rings(const Ring4Args& a, int lat0, int inst, int tid, float2* sm, float* s_rw,
                                             Sync sync) {
    using C = R4<M2>;
    constexpr int M = 24 * M2, A = C::A, B = M2 / A, P1 = C::P1, Bp = C::Bp, Q = C::Q, RING = C::RING;
    constexpr int G = 128 / M2, GP = G / 2, B2 = B + 1;
    constexpr int TA = 24 / A, TB = 24 / B;
    constexpr int NT = 256;
    static_assert(B > 1, "the wide ring transform exchanges pass-2b tiles");
    const float2* __restrict__ tw1 = a.ftw;
    const float2* __restrict__ tw2 = tw1 + 24 * P1;
    float2* buf = sm;
    const int N = a.N, nlat = a.nlat, ld = N + 1;
    const float2* gs = a.gsyn + size_t(inst) * a.sgs;
    float2* ga = a.gana + size_t(inst) * a.sga;

    // stage the spectra as in ring4_rings, 256 threads
    constexpr int NLD = (3 * 8 * M2 * GP + NT - 1) / NT;
    int m0 = tid, fr0 = 0;
    while (m0 >= ld) {
        m0 -= ld;
        ++fr0;
    }
    float4 stv[NLD];
    {
        int m = m0, fr = fr0;
#pragma unroll
        for (int k = 0; k < NLD; ++k) {
            const int rp = fr % GP, f = fr / GP;
            const int pr = lat0 / 2 + rp;
            stv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (f < 3 && 2 * pr < nlat)
                stv[k] = __ldcg(reinterpret_cast<const float4*>(gs + gsyn_index(a.pairs, f, m, 2 * pr, N, nlat)));
            m += NT;
            while (m >= ld) {
                m -= ld;
                ++fr;
            }
        }
    }
    sync();
    const int h = tid / 128, u = tid % 128, r = u / M2, t = u % M2;
    const int lat = lat0 + r;
    const float fc = lat < nlat ? a.two_omega * float(a.x[lat]) : 0.f;
    if (tid < G) s_rw[tid] = lat0 + tid < nlat ? float(a.rw[lat0 + tid]) : 0.f;
    {
        int m = m0, fr = fr0;
#pragma unroll
        for (int k = 0; k < NLD; ++k) {
            const int rp = fr % GP, f = fr / GP;
            if (f < 3) {
                buf[(2 * rp) * RING + f * ld + m] = make_float2(stv[k].x, stv[k].y);
                buf[(2 * rp + 1) * RING + f * ld + m] = make_float2(stv[k].z, stv[k].w);
            }
            m += NT;
            while (m >= ld) {
                m -= ld;
                ++fr;
            }
        }
    }
    sync();
    float2* XA = buf + r * RING;
    float2* XB = buf + (G + r) * RING;
    float2* X = h ? XB : XA;

    // pass 1: A = zeta + i u_theta (h = 0) or B = u_phi (h = 1)
    cx<float> x[24];
#pragma unroll
    for (int n1 = 0; n1 < 24; ++n1) {
        const int n = t + M2 * n1;
        cx<float> z{0.f, 0.f};
        if (n1 >= 8 && n1 < 16) {
        } else if (n <= N) {
            if (h == 0) {
                float2 g0 = XA[n], g1 = XA[ld + n];
                if (n == 0) g0.y = g1.y = 0.f;
                z = {g0.x - g1.y, g0.y + g1.x};
            } else {
                const float2 g2 = XA[2 * ld + n];
                z = {g2.x, n == 0 ? 0.f : g2.y};
            }
        } else if (n >= M - N) {
            const int mm = M - n;
            if (h == 0) {
                const float2 g0 = XA[mm], g1 = XA[ld + mm];
                z = {g0.x + g1.y, g1.x - g0.y};
            } else {
                const float2 g2 = XA[2 * ld + mm];
                z = {g2.x, -g2.y};
            }
        }
        x[n1] = z;
    }
    dft24<+1>(x);
#pragma unroll
    for (int k1 = 1; k1 < 24; ++k1) x[k1] = cmul(x[k1], ldg2(&tw1[k1 * P1 + t]));
    sync();
#pragma unroll
    for (int k1 = 0; k1 < 24; ++k1) st2(&X[k1 * P1 + t], x[k1]);
    sync();

    // pass 2a: task (k1 = j A + kq, b) of this thread's signal
    const int b = t % B, kq = t / B;
    {
    cx<float> uu[TA][A];
#pragma unroll
    for (int j = 0; j < TA; ++j) {
        const int k1 = j * A + kq;
#pragma unroll
        for (int ap = 0; ap < A; ++ap) uu[j][ap] = ld2(&X[k1 * P1 + b + B * ap]);
        dftn<A>(uu[j], +1);
#pragma unroll
        for (int c = 1; c < A; ++c) uu[j][c] = cmul(uu[j][c], ldg2(&tw2[c * B2 + b]));
    }
    sync();
#pragma unroll
    for (int j = 0; j < TA; ++j) {
        const int k1 = j * A + kq;
#pragma unroll
        for (int c = 0; c < A; ++c) st2(&X[k1 * Q + c * Bp + b], uu[j][c]);
    }
    }
    sync();
    // pass 2b: task (k1 = j B + kq2, c); the B threads store their values
    // back where they read them
    const int c = C::SW ? t / B : t % A, kq2 = C::SW ? t % B : t / A;
    cx<float> v[TB][B];
#pragma unroll
    for (int j = 0; j < TB; ++j) {
        const int k1 = j * B + kq2;
#pragma unroll
        for (int bb = 0; bb < B; ++bb) v[j][bb] = ld2(&X[k1 * Q + c * Bp + bb]);
        dftn<B>(v[j], +1);
        if (h == 1) {
#pragma unroll
            for (int bb = 0; bb < B; ++bb) st2(&X[k1 * Q + c * Bp + bb], v[j][bb]);
        }
    }
    sync();
    if (h == 0) {
#pragma unroll
        for (int j = 0; j < TB; ++j) {
            const int k1 = j * B + kq2;
#pragma unroll
            for (int d = 0; d < B; ++d) {
                // zeta = Re A, u_theta = Im A, u_phi = Re B;  W = (-q u_phi, q u_theta)
                const cx<float> zb = ld2(&XB[k1 * Q + c * Bp + d]);
                const float q = v[j][d].x + fc;
                v[j][d] = {-q * zb.x, q * v[j][d].y};
            }
            dftn<B>(v[j], -1);
#pragma unroll
            for (int bb = 1; bb < B; ++bb) v[j][bb] = cmul(v[j][bb], conjg2(&tw2[c * B2 + bb]));
#pragma unroll
            for (int bb = 0; bb < B; ++bb) st2(&XA[k1 * Q + c * Bp + bb], v[j][bb]);
        }
    }
    sync();
    // the B buffers are free from here: the remaining passes alternate
    // between XA and XB, so each needs one barrier
    if (h == 0) {
        // A-point DFT over c -> a', twiddle e^{-2 pi i t k1 / M} with t = b + B a'
#pragma unroll
        for (int j = 0; j < TA; ++j) {
            const int k1 = j * A + kq;
            cx<float> y[A];
#pragma unroll
            for (int cc = 0; cc < A; ++cc) y[cc] = ld2(&XA[k1 * Q + cc * Bp + b]);
            dftn<A>(y, -1);
#pragma unroll
            for (int ap = 0; ap < A; ++ap) st2(&XB[k1 * P1 + b + B * ap], cmul(y[ap], conjg2(&tw1[k1 * P1 + b + B * ap])));
        }
    }
    sync();
    // 24-point DFT over k1 -> W's spectrum at n = t + M2 n1 (only m <= N and
    // m >= M - N are read back: n1 = 8 .. 15 are never needed)
    if (h == 0) {
        cx<float> y[24];
#pragma unroll
        for (int k1 = 0; k1 < 24; ++k1) y[k1] = ld2(&XB[k1 * P1 + t]);
        dft24<-1>(y);
#pragma unroll
        for (int n1 = 0; n1 < 24; ++n1)
            if (n1 < 8 || n1 >= 16) st2(&XA[t + M2 * n1], y[n1]);
    }
    sync();

    // separate the two real fields, truncate to m <= N, weight, store
    for (int i = tid; i < ld * GP; i += NT) {
        const int rp = i % GP, m = i / GP;
        const int l = lat0 + 2 * rp;
        if (l >= nlat) continue;
        float4 oA, oB;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float2* Z = buf + (2 * rp + e) * RING;
            const float2 p = Z[m], q = Z[(M - m) % M];
            const float sc = s_rw[2 * rp + e];
            const float ax = 0.5f * (p.x + q.x) * sc, ay = 0.5f * (p.y - q.y) * sc;
            const float bx = 0.5f * (p.y + q.y) * sc, by = 0.5f * (q.x - p.x) * sc;
            if (e == 0) {
                oA.x = ax; oA.y = ay; oB.x = bx; oB.y = by;
            } else {
                oA.z = ax; oA.w = ay; oB.z = bx; oB.w = by;
            }
        }
        *reinterpret_cast<float4*>(ga + size_t(m) * nlat + l) = oA;
        *reinterpret_cast<float4*>(ga + size_t(ld + m) * nlat + l) = oB;
    }
}

}  // namespace sph
