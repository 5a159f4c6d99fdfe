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

#include "internal.h"

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
    k_ring<T, TW, MODE><<<dim3(P->nlat, nb), threads, sm, P->stream>>>(a, P->fft, tw);
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
    a.two_omega = 2.0 * P->Omega;
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
// Tiled transposes between the order-major layout of the Legendre kernels
// ([f][m][row]) and the latitude-major layout of the ring kernel
// ([f][row][m]); 32 x 32 complex tiles through shared memory, both sides
// coalesced.

template <typename C>
__global__ void __launch_bounds__(256) k_transpose(const C* __restrict__ in, C* __restrict__ out, int R, int Cn) {
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
        k_transpose<double2><<<grd, blk, 0, P->stream>>>(reinterpret_cast<const double2*>(in),
                                                          reinterpret_cast<double2*>(out), R, Cn);
    else
        k_transpose<float2><<<grd, blk, 0, P->stream>>>(reinterpret_cast<const float2*>(in),
                                                         reinterpret_cast<float2*>(out), R, Cn);
    stage_end(P, SPHNSE_STAGE_TRANSPOSE);
    return check_cuda(cudaGetLastError());
}

}  // namespace sph
