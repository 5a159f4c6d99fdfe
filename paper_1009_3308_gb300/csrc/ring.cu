// Longitude ("ring") kernel: one CTA per Gauss latitude theta_p.
//
// RHS mode (Sec. 4.2: the phi sums of Eqs. (app_soln_rep), (eval_nonlin1)
// are Fourier sums, evaluated by FFT):
//   1. inverse FFT of the Hermitian spectra g_m, |m| <= N (zero-padded to M):
//      z1 = zeta + i u_theta, z2 = u_phi              (two complex M-point FFTs)
//   2. pointwise product (Eqs. (short_nonlin1), (C)):
//      q = zeta + 2 Omega cos(theta_p),  W_theta = -q u_phi,  W_phi = q u_theta
//   3. forward FFT of W_theta + i W_phi, separation of the two real spectra,
//      truncation to m = 0..N, scaling by (2 pi / M) w_p / sin(theta_p)
//      (the quadrature weight of Eq. (quadrule) and the 1/sin of the basis).
// M = nlon = 2^a 3^b; Stockham autosort radix-8/4/2/3 stages in shared memory
// (radix 3 last, so every stride Ns before it is a power of two), FP64
// twiddles e^{-2 pi i t / M} from the host (FP32 copy for FP32 mode) staged in
// shared memory.
// Products keep |m| <= 2N and M >= 3N + 2 > 3N, so the truncated m <= N
// coefficients are alias-free.
//
// Other modes reuse the same machinery: GRID writes zeta, u_theta, u_phi to
// grid rows; PROJECT transforms given grid rows of a tangential field;
// ADJOINT evaluates the transposed linearised product (see rhs_adjoint).
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"
#include "ptx.cuh"

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

// One in-place Stockham stage of radix R over NSIG signals (buf[s], M points):
// every thread first reads and transforms all of its butterflies into
// registers, the block synchronises, then writes them to their autosorted
// positions.  Ns = product of the earlier radices; nsh = log2(Ns) when Ns is
// a power of two (radix-3 stages run last, so this holds unless M has 3^2).
// The launch uses blockDim >= M/6, so a thread owns at most MAXB butterflies.
template <typename T, typename TW, int R, int NSIG>
__device__ __forceinline__ void stage(cx<T>* const* buf, int M, int Ns, int nsh, const TW* tw, int sign) {
    constexpr int MAXB = R == 2 ? 3 : (R == 8 ? 1 : 2);
    const int nb = M / R;
    const int twstride = M / (Ns * R);
    cx<T> v[NSIG][MAXB][R];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int j = threadIdx.x + b * blockDim.x;
        if (j < nb) {
            const int k = nsh >= 0 ? (j & (Ns - 1)) : (j % Ns);
            cx<T> w[R];
#pragma unroll
            for (int r = 1; r < R; ++r) w[r] = twiddle<T>(tw, k * r * twstride, sign);
#pragma unroll
            for (int sg = 0; sg < NSIG; ++sg) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const cx<T> a = buf[sg][j + r * nb];
                    v[sg][b][r] = r == 0 ? a : cmul(a, w[r]);
                }
                dft<T, R>(v[sg][b], sign);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int j = threadIdx.x + b * blockDim.x;
        if (j < nb) {
            const int k = nsh >= 0 ? (j & (Ns - 1)) : (j % Ns);
            const int q = nsh >= 0 ? (j >> nsh) : (j / Ns);
            const int idx = q * Ns * R + k;
#pragma unroll
            for (int sg = 0; sg < NSIG; ++sg)
#pragma unroll
                for (int r = 0; r < R; ++r) buf[sg][idx + r * Ns] = v[sg][b][r];
        }
    }
    __syncthreads();
}

// Full M-point transform (sign -1 forward, +1 inverse) of NSIG signals in place.
template <typename T, typename TW, int NSIG>
__device__ void fft(cx<T>* const* buf, const FFTPlan& plan, const TW* tw, int sign) {
    const int M = plan.n;
    int Ns = 1;
    for (int st = 0; st < plan.nstages; ++st) {
        const int R = plan.radix[st];
        const int nsh = (Ns & (Ns - 1)) == 0 ? __ffs(Ns) - 1 : -1;
        if (R == 8) stage<T, TW, 8, NSIG>(buf, M, Ns, nsh, tw, sign);
        else if (R == 4) stage<T, TW, 4, NSIG>(buf, M, Ns, nsh, tw, sign);
        else if (R == 2) stage<T, TW, 2, NSIG>(buf, M, Ns, nsh, tw, sign);
        else stage<T, TW, 3, NSIG>(buf, M, Ns, nsh, tw, sign);
        Ns *= R;
    }
}

struct RingArgs {
    int N, M, nlat, mode;
    double two_omega;
    const double* x;       // cos(theta)
    const double* s;       // sin(theta)
    const double* rw;      // (2 pi / M) w_p / sin(theta_p)
    const void* gsyn;      // [nf][nlat][N+1] complex T (row-major)
    void* gana;            // [nf][nlat][N+1] complex T (row-major)
    const double* gin0;    // grid input rows (PROJECT)
    const double* gin1;
    double* gout0;         // grid output rows (GRID)
    double* gout1;
    double* gout2;
    size_t sgs, sga;       // per-instance strides (complex entries) along gridDim.y
};

template <typename T, typename TW, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_ring(RingArgs a, FFTPlan plan, const TW* __restrict__ tw) {
    pdl_launch();
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NBUF = MODE == RING_ADJOINT ? 3 : (MODE == RING_PROJECT ? 1 : 2);
    cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
    // the twiddle table e^{-2 pi i t / M} lives in shared memory after the buffers
    T* tws = reinterpret_cast<T*>(buf + NBUF * a.M);
    for (int t = threadIdx.x; t < 2 * a.M; t += blockDim.x) tws[t] = T(tw[t]);
    const int row = blockIdx.x;
    const int M = a.M, N = a.N, nlat = a.nlat;
    const size_t ld = size_t(N + 1);
    const cx<T>* gs = reinterpret_cast<const cx<T>*>(a.gsyn) + size_t(blockIdx.y) * a.sgs;
    cx<T>* ga = reinterpret_cast<cx<T>*>(a.gana) + size_t(blockIdx.y) * a.sga;
    auto G = [&](int f, int m) -> cx<T> { return gs[(size_t(f) * nlat + row) * ld + m]; };

    cx<T>* src[3] = {buf, buf + M, buf + 2 * M};

    if constexpr (MODE != RING_PROJECT) {
        // Hermitian spectra of two real fields packed as a + i b:
        //   Z_m = g^a_m + i g^b_m (m <= N);  Z_{M-m} = conj(g^a_m) + i conj(g^b_m)
        const int nsig = MODE == RING_ADJOINT ? 3 : 2;
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            int mm = -1;
            bool upper = false;
            if (m <= N) mm = m;
            else if (m >= M - N) { mm = M - m; upper = true; }
            for (int sgi = 0; sgi < nsig; ++sgi) {
                // fields packed per signal: RHS/GRID (0,1),(2,-); ADJOINT (0,1),(2,3),(4,-)
                const int fa = 2 * sgi, fb = 2 * sgi + 1;
                const bool has_b = (MODE == RING_ADJOINT) ? fb <= 4 : fb <= 2;
                cx<T> z{T(0), T(0)};
                if (mm >= 0) {
                    cx<T> ga_ = G(fa, mm);
                    cx<T> gb_ = has_b ? G(fb, mm) : cx<T>{T(0), T(0)};
                    if (mm == 0) { ga_.y = T(0); gb_.y = T(0); }
                    if (!upper) z = {ga_.x - gb_.y, ga_.y + gb_.x};
                    else        z = {ga_.x + gb_.y, gb_.x - ga_.y};
                }
                src[sgi][m] = z;
            }
        }
        __syncthreads();
        fft<T, T, MODE == RING_ADJOINT ? 3 : 2>(src, plan, tws, +1);
    }

    if constexpr (MODE == RING_GRID) {
        for (int q = threadIdx.x; q < M; q += blockDim.x) {
            if (a.gout0) a.gout0[size_t(row) * M + q] = double(src[0][q].x);
            if (a.gout1) a.gout1[size_t(row) * M + q] = double(src[0][q].y);
            if (a.gout2) a.gout2[size_t(row) * M + q] = double(src[1][q].x);
        }
        return;
    }

    constexpr int nout = MODE == RING_ADJOINT ? 2 : 1;
    if constexpr (MODE == RING_RHS) {
        const T fc = T(a.two_omega * a.x[row]);
        for (int q = threadIdx.x; q < M; q += blockDim.x) {
            const T zeta = src[0][q].x, uth = src[0][q].y, uph = src[1][q].x;
            const T qq = zeta + fc;
            src[0][q] = {-qq * uph, qq * uth};
        }
    } else if constexpr (MODE == RING_PROJECT) {
        for (int q = threadIdx.x; q < M; q += blockDim.x)
            src[0][q] = {T(a.gin0[size_t(row) * M + q]), T(a.gin1[size_t(row) * M + q])};
    } else {  // RING_ADJOINT: fields zeta, u_th, u_ph, v_th, v_ph
        const T fc = T(a.two_omega * a.x[row]);
        for (int q = threadIdx.x; q < M; q += blockDim.x) {
            const T zeta = src[0][q].x, uth = src[0][q].y;
            const T uph = src[1][q].x, vth = src[1][q].y, vph = src[2][q].x;
            const T qq = zeta + fc;
            // X = -q xhat x v = (q v_phi, -q v_theta); rho = v . (xhat x u) = -v_th u_ph + v_ph u_th
            src[0][q] = {qq * vph, -qq * vth};
            src[1][q] = {-vth * uph + vph * uth, T(0)};
        }
    }
    __syncthreads();
    fft<T, T, nout>(src, plan, tws, -1);

    const T scale = T(a.rw[row]);
    for (int m = threadIdx.x; m <= N; m += blockDim.x) {
        const cx<T> p = src[0][m];
        const cx<T> r = src[0][(M - m) % M];
        // W = A + i B with A, B real fields: A_m = (Z_m + conj Z_{M-m}) / 2,
        // B_m = (Z_m - conj Z_{M-m}) / (2 i)
        cx<T> A{T(0.5) * (p.x + r.x), T(0.5) * (p.y - r.y)};
        cx<T> B{T(0.5) * (p.y + r.y), T(0.5) * (r.x - p.x)};
        ga[(size_t(0) * nlat + row) * ld + m] = {A.x * scale, A.y * scale};
        ga[(size_t(1) * nlat + row) * ld + m] = {B.x * scale, B.y * scale};
        if constexpr (nout == 2) {
            // scalar field rho: plain quadrature weight (2 pi / M) w_p
            const T sc2 = scale * T(a.s[row]);
            const cx<T> z = src[1][m];
            ga[(size_t(2) * nlat + row) * ld + m] = {z.x * sc2, z.y * sc2};
        }
    }
}

template <typename T, typename TW, int MODE>
static void ring_t(sphnse_plan* P, const RingArgs& a, const TW* tw, int threads, int nb = 1) {
    const int nbuf = MODE == RING_ADJOINT ? 3 : (MODE == RING_PROJECT ? 1 : 2);
    const size_t sm = size_t(nbuf) * P->nlon * sizeof(cx<T>) + size_t(P->nlon) * 2 * sizeof(T);
    cudaFuncSetAttribute(k_ring<T, TW, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    launch_pdl_small(P->n_cta, k_ring<T, TW, MODE>, dim3(P->nlat, nb), dim3(threads), sm, P->stream, a, P->fft, tw);
}

// FP32 RHS ring pass over nb instances (latitude-major buffers with strides)
int launch_ring_batch(sphnse_plan* P, int nb, const float* gsyn_r, size_t sgs, float* gana_r, size_t sga) {
    RingArgs a{};
    a.N = P->N;
    a.M = P->nlon;
    a.nlat = P->nlat;
    a.mode = RING_RHS;
    a.two_omega = 2.0 * P->Omega;
    a.x = P->d_x;
    a.s = P->d_s;
    a.rw = P->d_rw;
    a.gsyn = gsyn_r;
    a.gana = gana_r;
    a.sgs = sgs / 2;
    a.sga = sga / 2;
    int threads = ((P->nlon / 6 + 31) / 32) * 32;
    if (threads < 32) threads = 32;
    stage_begin(P, SPHNSE_STAGE_RING);
    ring_t<float, float, RING_RHS>(P, a, P->d_tw32, threads, nb);
    stage_end(P, SPHNSE_STAGE_RING);
    return check_cuda(cudaGetLastError());
}

template <typename T, typename TW>
static void ring_mode(sphnse_plan* P, int mode, const RingArgs& a, const TW* tw, int threads) {
    switch (mode) {
        case RING_RHS: ring_t<T, TW, RING_RHS>(P, a, tw, threads); break;
        case RING_GRID: ring_t<T, TW, RING_GRID>(P, a, tw, threads); break;
        case RING_PROJECT: ring_t<T, TW, RING_PROJECT>(P, a, tw, threads); break;
        default: ring_t<T, TW, RING_ADJOINT>(P, a, tw, threads); break;
    }
}

int launch_ring(sphnse_plan* P, int mode, int prec, const double* gin0, const double* gin1,
                double* gout0, double* gout1, double* gout2) {
    RingArgs a;
    a.N = P->N;
    a.M = P->nlon;
    a.nlat = P->nlat;
    a.mode = mode;
    a.two_omega = mode == RING_RHS && P->coriolis_split ? 0.0 : 2.0 * P->Omega;
    a.x = P->d_x;
    a.s = P->d_s;
    a.rw = P->d_rw;
    a.gsyn = P->d_gsyn_r;
    a.gana = P->d_gana_r;
    a.gin0 = gin0;
    a.gin1 = gin1;
    a.gout0 = gout0;
    a.gout1 = gout1;
    a.gout2 = gout2;
    a.sgs = a.sga = 0;
    // in-place stages need blockDim >= M / 6 (at most 3 butterflies per thread)
    int threads = ((P->nlon / 6 + 31) / 32) * 32;
    if (threads < 32) threads = 32;
    stage_begin(P, SPHNSE_STAGE_RING);
    if (prec == SPHNSE_FP64) ring_mode<double, double>(P, mode, a, P->d_tw, threads);
    else ring_mode<float, float>(P, mode, a, P->d_tw32, threads);
    stage_end(P, SPHNSE_STAGE_RING);
    return check_cuda(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Four-step ring kernel for M = 24 M2 (M2 = 4 .. 64), FP32, RHS mode, reading
// the synthesis output (order-major or latitude-pair-major) and writing the
// order-major spectra of the analysis directly, without transposes.
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
// One CTA of 128 threads holds G = 128 / M2 consecutive rings, so every
// order-major access moves G consecutive latitudes (>= 16 bytes).

template <int M2> struct R4;
template <> struct R4<64> { static constexpr int A = 8, P1 = 72, Bp = 9, Q = 72, RING = 1728; };
template <> struct R4<32> { static constexpr int A = 8, P1 = 36, Bp = 5, Q = 40, RING = 960; };
template <> struct R4<16> { static constexpr int A = 4, P1 = 20, Bp = 5, Q = 20, RING = 480; };
template <> struct R4<8> { static constexpr int A = 8, P1 = 9, Bp = 1, Q = 9, RING = 216; };
template <> struct R4<4> { static constexpr int A = 4, P1 = 5, Bp = 1, Q = 5, RING = 124; };

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

template <int M2>
__global__ void __launch_bounds__(128, 3) k_ring4(Ring4Args a) {
    using C = R4<M2>;
    constexpr int M = 24 * M2, A = C::A, B = M2 / A, P1 = C::P1, Bp = C::Bp, Q = C::Q, RING = C::RING;
    constexpr int G = 128 / M2, GP = G / 2, B2 = B + 1;
    constexpr int TA = 24 / A, TB = 24 / B;
    extern __shared__ __align__(16) float2 sm4[];
    float2* tw1 = sm4;
    float2* tw2 = tw1 + 24 * P1;
    float2* buf = tw2 + ((A * B2 + 1) & ~1);
    // twiddles do not depend on the predecessor: stage them before waiting for it,
    // with all of a thread's loads issued before its stores
    constexpr int NTW = (24 * P1 + A * B2 + 127) / 128;
    {
        float2 tv[NTW];
#pragma unroll
        for (int k = 0; k < NTW; ++k) {
            const int i = threadIdx.x + 128 * k;
            tv[k] = i < 24 * P1 + A * B2 ? __ldg(a.ftw + i) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < NTW; ++k) {
            const int i = threadIdx.x + 128 * k;
            if (i < 24 * P1 + A * B2) tw1[i] = tv[k];
        }
    }
    pdl_launch();
    pdl_wait();
    const int N = a.N, nlat = a.nlat, ld = N + 1;
    const int lat0 = blockIdx.x * G;
    const float2* gs = a.gsyn + size_t(blockIdx.y) * a.sgs;
    float2* ga = a.gana + size_t(blockIdx.y) * a.sga;

    // stage the spectra: ring r, field f, order m -> buf[r RING + f (N+1) + m].
    // In the latitude-pair-major input, [f][row / 2][m][row % 2], the CTA's
    // pairs are contiguous runs of (N+1) float4 per field; the order-major
    // input gives one float4 per (f, m).  3 (N+1) G / 2 <= 1536 float4 loads
    // per CTA, all of a thread's issued before its stores.
    constexpr int NLD = (3 * 8 * M2 * GP + 127) / 128;
    float4 stv[NLD];
#pragma unroll
    for (int k = 0; k < NLD; ++k) {
        const int i = threadIdx.x + 128 * k;
        const int m = i % ld, fr = i / ld, rp = fr % GP, f = fr / GP;
        const int pr = lat0 / 2 + rp;
        stv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < 3 * ld * GP && 2 * pr < nlat)
            stv[k] = __ldcs(reinterpret_cast<const float4*>(gs + gsyn_index(a.pairs, f, m, 2 * pr, N, nlat)));
    }
    const int r = threadIdx.x / M2, t = threadIdx.x % M2;
    const int lat = lat0 + r;
    const float fc = lat < nlat ? a.two_omega * float(a.x[lat]) : 0.f;
    __shared__ float s_rw[G];
    if (threadIdx.x < G) s_rw[threadIdx.x] = lat0 + int(threadIdx.x) < nlat ? float(a.rw[lat0 + threadIdx.x]) : 0.f;
#pragma unroll
    for (int k = 0; k < NLD; ++k) {
        const int i = threadIdx.x + 128 * k;
        if (i < 3 * ld * GP) {
            const int m = i % ld, fr = i / ld, rp = fr % GP, f = fr / GP;
            buf[(2 * rp) * RING + f * ld + m] = make_float2(stv[k].x, stv[k].y);
            buf[(2 * rp + 1) * RING + f * ld + m] = make_float2(stv[k].z, stv[k].w);
        }
    }
    __syncthreads();
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
        const cx<float> w = ld2(&tw1[k1 * P1 + t]);
        xa[k1] = cmul(xa[k1], w);
        xb[k1] = cmul(xb[k1], w);
    }
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < 24; ++k1) {
        st2(&XA[k1 * P1 + t], xa[k1]);
        st2(&XB[k1 * P1 + t], xb[k1]);
    }
    __syncthreads();

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
                const cx<float> w = ld2(&tw2[c * B2 + b]);
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

    if constexpr (B > 1) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < TA; ++j) {
            const int k1 = j * A + kq;
#pragma unroll
            for (int c = 0; c < A; ++c) {
                st2(&XA[k1 * Q + c * Bp + b], ua[j][c]);
                st2(&XB[k1 * Q + c * Bp + b], ub[j][c]);
            }
        }
        __syncthreads();
        // pass 2b: task (k1 = j B + kq2, c) -> X[k1 + 24 (c + A d)]
        const int c = t % A, kq2 = t / A;
        cx<float> va[TB][B], vb[TB][B];
#pragma unroll
        for (int j = 0; j < TB; ++j) {
            const int k1 = j * B + kq2;
#pragma unroll
            for (int bb = 0; bb < B; ++bb) {
                va[j][bb] = ld2(&XA[k1 * Q + c * Bp + bb]);
                vb[j][bb] = ld2(&XB[k1 * Q + c * Bp + bb]);
            }
            dftn<B>(va[j], +1);
            dftn<B>(vb[j], +1);
#pragma unroll
            for (int d = 0; d < B; ++d) product(va[j][d], vb[j][d]);
            // forward, backwards through the factorisation: B-point DFT over d
            dftn<B>(va[j], -1);
#pragma unroll
            for (int bb = 1; bb < B; ++bb) va[j][bb] = cmul(va[j][bb], conjf2(tw2[c * B2 + bb]));
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < TB; ++j) {
            const int k1 = j * B + kq2;
#pragma unroll
            for (int bb = 0; bb < B; ++bb) st2(&XA[k1 * Q + c * Bp + bb], va[j][bb]);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < TA; ++j) {
            const int k1 = j * A + kq;
#pragma unroll
            for (int cc = 0; cc < A; ++cc) ua[j][cc] = ld2(&XA[k1 * Q + cc * Bp + b]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < TA; ++j)
#pragma unroll
            for (int cc = 0; cc < A; ++cc) product(ua[j][cc], ub[j][cc]);
    }
    // A-point DFT over c -> a', twiddle e^{-2 pi i t k1 / M} with t = b + B a'
#pragma unroll
    for (int j = 0; j < TA; ++j) {
        const int k1 = j * A + kq;
        dftn<A>(ua[j], -1);
#pragma unroll
        for (int ap = 0; ap < A; ++ap) ua[j][ap] = cmul(ua[j][ap], conjf2(tw1[k1 * P1 + b + B * ap]));
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TA; ++j) {
        const int k1 = j * A + kq;
#pragma unroll
        for (int ap = 0; ap < A; ++ap) st2(&XA[k1 * P1 + b + B * ap], ua[j][ap]);
    }
    __syncthreads();
    // 24-point DFT over k1 -> W's spectrum at n = t + M2 n1
    cx<float> y[24];
#pragma unroll
    for (int k1 = 0; k1 < 24; ++k1) y[k1] = ld2(&XA[k1 * P1 + t]);
    dft24<-1>(y);
    __syncthreads();
    // only m <= N and m >= M - N are read back: n1 = 8 .. 15 are never needed
#pragma unroll
    for (int n1 = 0; n1 < 24; ++n1)
        if (n1 < 8 || n1 >= 16) st2(&XA[t + M2 * n1], y[n1]);
    __syncthreads();

    // separate the two real fields, truncate to m <= N, weight, store
    for (int i = threadIdx.x; i < ld * GP; i += 128) {
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

template <int M2>
static constexpr size_t ring4_smem() {
    using C = R4<M2>;
    constexpr int A = C::A, B = M2 / A, G = 128 / M2;
    return (size_t(24) * C::P1 + ((A * (B + 1) + 1) & ~1) + size_t(2) * G * C::RING) * sizeof(float2);
}

template <int M2>
static int ring4_t(sphnse_plan* P, int nb, const float* gsyn, size_t sgs, float* gana, size_t sga, int pairs) {
    constexpr size_t sm = ring4_smem<M2>();
    static_assert(sm <= 227 * 1024, "ring4 shared memory");
    cudaFuncSetAttribute(k_ring4<M2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    Ring4Args a;
    a.N = P->N;
    a.nlat = P->nlat;
    a.two_omega = P->coriolis_split ? 0.f : float(2.0 * P->Omega);
    a.x = P->d_x;
    a.rw = P->d_rw;
    a.gsyn = reinterpret_cast<const float2*>(gsyn);
    a.gana = reinterpret_cast<float2*>(gana);
    a.ftw = reinterpret_cast<const float2*>(P->d_ftw);
    a.sgs = sgs / 2;
    a.sga = sga / 2;
    a.pairs = pairs;
    constexpr int G = 128 / M2;
    return check_cuda(launch_pdl(k_ring4<M2>, dim3((P->nlat + G - 1) / G, nb), dim3(128), sm, P->stream, a));
}

int ring4_m2(int nlon, int nlat) {
    if (nlon % 24 || nlat % 2) return 0;
    const int M2 = nlon / 24;
    return (M2 == 4 || M2 == 8 || M2 == 16 || M2 == 32 || M2 == 64) ? M2 : 0;
}

bool ring4_ok(const sphnse_plan* P) { return ring4_m2(P->nlon, P->nlat) != 0 && P->d_ftw != nullptr; }

// twiddle tables of the four-step kernel (FP64 -> FP32), in its padded layout
std::vector<float> ring4_twiddles(int nlon) {
    const int M2 = ring4_m2(nlon, 2);
    if (!M2) return {};
    int A = 0, P1 = 0;
    switch (M2) {
        case 64: A = R4<64>::A; P1 = R4<64>::P1; break;
        case 32: A = R4<32>::A; P1 = R4<32>::P1; break;
        case 16: A = R4<16>::A; P1 = R4<16>::P1; break;
        case 8: A = R4<8>::A; P1 = R4<8>::P1; break;
        default: A = R4<4>::A; P1 = R4<4>::P1; break;
    }
    const int B = M2 / A, B2 = B + 1;
    std::vector<float> tw(2 * (size_t(24) * P1 + size_t(A) * B2), 0.f);
    for (int k1 = 0; k1 < 24; ++k1)
        for (int t = 0; t < M2; ++t) {
            const double ang = 2.0 * M_PI * double((long(t) * k1) % nlon) / double(nlon);
            tw[2 * (k1 * P1 + t)] = float(std::cos(ang));
            tw[2 * (k1 * P1 + t) + 1] = float(std::sin(ang));
        }
    float* t2 = tw.data() + 2 * 24 * P1;
    for (int c = 0; c < A; ++c)
        for (int bb = 0; bb < B; ++bb) {
            const double ang = 2.0 * M_PI * double((bb * c) % M2) / double(M2);
            t2[2 * (c * B2 + bb)] = float(std::cos(ang));
            t2[2 * (c * B2 + bb) + 1] = float(std::sin(ang));
        }
    return tw;
}

// FP32 RHS ring pass over nb instances, order-major buffers
int launch_ring4(sphnse_plan* P, int nb, const float* gsyn, size_t sgs, float* gana, size_t sga, int pairs) {
    stage_begin(P, SPHNSE_STAGE_RING);
    int rc;
    switch (ring4_m2(P->nlon, P->nlat)) {
        case 64: rc = ring4_t<64>(P, nb, gsyn, sgs, gana, sga, pairs); break;
        case 32: rc = ring4_t<32>(P, nb, gsyn, sgs, gana, sga, pairs); break;
        case 16: rc = ring4_t<16>(P, nb, gsyn, sgs, gana, sga, pairs); break;
        case 8: rc = ring4_t<8>(P, nb, gsyn, sgs, gana, sga, pairs); break;
        case 4: rc = ring4_t<4>(P, nb, gsyn, sgs, gana, sga, pairs); break;
        default: rc = SPHNSE_E_UNSUPPORTED;
    }
    stage_end(P, SPHNSE_STAGE_RING);
    return rc;
}

// ---------------------------------------------------------------------------
// Tiled transposes between the order-major layout of the Legendre kernels
// ([f][m][row]) and the latitude-major layout of the ring kernel
// ([f][row][m]); 32 x 32 complex tiles through shared memory, both sides
// coalesced.

template <typename C>
__global__ void __launch_bounds__(256) k_transpose(const C* __restrict__ in, C* __restrict__ out, int R, int Cn) {
    // no early trigger: several waves at large sizes (see k_prep)
    pdl_wait();
    __shared__ C tile[32][33];
    const int f = blockIdx.z;
    const C* src = in + size_t(f) * R * Cn;
    C* dst = out + size_t(f) * R * Cn;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < Cn) tile[i][threadIdx.x] = src[size_t(r) * Cn + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < Cn) dst[size_t(c) * R + r] = tile[threadIdx.x][i];
    }
}

// in: [nf][R][Cn] -> out: [nf][Cn][R]
int launch_transpose(sphnse_plan* P, const void* in, void* out, int R, int Cn, int nf, int prec) {
    dim3 blk(32, 8), grd((Cn + 31) / 32, (R + 31) / 32, nf);
    stage_begin(P, SPHNSE_STAGE_TRANSPOSE);
    if (prec == SPHNSE_FP64)
        launch_pdl_small(P->n_cta, k_transpose<double2>, grd, blk, 0, P->stream, reinterpret_cast<const double2*>(in),
                   reinterpret_cast<double2*>(out), R, Cn);
    else
        launch_pdl_small(P->n_cta, k_transpose<float2>, grd, blk, 0, P->stream, reinterpret_cast<const float2*>(in),
                   reinterpret_cast<float2*>(out), R, Cn);
    stage_end(P, SPHNSE_STAGE_TRANSPOSE);
    return check_cuda(cudaGetLastError());
}

}  // namespace sph
