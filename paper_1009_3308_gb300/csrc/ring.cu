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
// M = nlon = 2^a 3^b; Stockham autosort radix-4/2/3 stages in shared memory,
// FP64 twiddles e^{-2 pi i t / M} from the host (FP32 copy for FP32 mode).
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

// Stockham autosort over nsig signals at once.  src[k]/dst[k] are the ping-pong
// buffers of signal k; on return src[k] holds the result.
template <typename T, typename TW>
__device__ void stockham(cx<T>** src, cx<T>** dst, int nsig, const FFTPlan& plan, const TW* tw, int sign) {
    const int M = plan.n;
    int Ns = 1;
    for (int st = 0; st < plan.nstages; ++st) {
        const int R = plan.radix[st];
        const int nb = M / R;
        const int twstride = M / (Ns * R);
        for (int j = threadIdx.x; j < nb; j += blockDim.x) {
            const int k = j % Ns;
            const int idx = (j / Ns) * Ns * R + k;
            for (int sgi = 0; sgi < nsig; ++sgi) {
                cx<T> v[4];
                for (int r = 0; r < R; ++r) {
                    cx<T> a = src[sgi][j + r * nb];
                    v[r] = r == 0 ? a : cmul(a, twiddle<T>(tw, k * r * twstride, sign));
                }
                if (R == 4) dft4(v, sign);
                else if (R == 2) dft2(v);
                else dft3(v, sign);
                for (int r = 0; r < R; ++r) dst[sgi][idx + r * Ns] = v[r];
            }
        }
        __syncthreads();
        for (int sgi = 0; sgi < nsig; ++sgi) {
            cx<T>* t = src[sgi];
            src[sgi] = dst[sgi];
            dst[sgi] = t;
        }
        Ns *= R;
    }
}

struct RingArgs {
    int N, M, nlat, mode;
    double two_omega;
    const double* x;       // cos(theta)
    const double* s;       // sin(theta)
    const double* rw;      // (2 pi / M) w_p / sin(theta_p)
    const void* gsyn;      // [nf][nlat][N+1] complex T
    void* gana;            // [nf][nlat][N+1] complex T
    const double* gin0;    // grid input rows (PROJECT)
    const double* gin1;
    double* gout0;         // grid output rows (GRID)
    double* gout1;
    double* gout2;
};

template <typename T, typename TW>
__global__ void __launch_bounds__(256) k_ring(RingArgs a, FFTPlan plan, const TW* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
    const int row = blockIdx.x;
    const int M = a.M, N = a.N, nlat = a.nlat;
    const size_t ld = size_t(N + 1);
    const cx<T>* gs = reinterpret_cast<const cx<T>*>(a.gsyn);
    cx<T>* ga = reinterpret_cast<cx<T>*>(a.gana);
    auto G = [&](int f, int m) -> cx<T> { return gs[(size_t(f) * nlat + row) * ld + m]; };

    cx<T>* src[3];
    cx<T>* dst[3];
    for (int k = 0; k < 3; ++k) {
        src[k] = buf + (2 * k) * M;
        dst[k] = buf + (2 * k + 1) * M;
    }

    if (a.mode != RING_PROJECT) {
        // Hermitian spectra of two real fields packed as a + i b:
        //   Z_m = g^a_m + i g^b_m (m <= N);  Z_{M-m} = conj(g^a_m) + i conj(g^b_m)
        const int nsig = a.mode == RING_ADJOINT ? 3 : 2;
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            int mm = -1;
            bool upper = false;
            if (m <= N) mm = m;
            else if (m >= M - N) { mm = M - m; upper = true; }
            for (int sgi = 0; sgi < nsig; ++sgi) {
                // fields packed per signal: RHS/GRID (0,1),(2,-); ADJOINT (0,1),(2,3),(4,-)
                const int fa = 2 * sgi, fb = 2 * sgi + 1;
                const bool has_b = (a.mode == RING_ADJOINT) ? fb <= 4 : fb <= 2;
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
        stockham<T, TW>(src, dst, nsig, plan, tw, +1);
    }

    if (a.mode == RING_GRID) {
        for (int q = threadIdx.x; q < M; q += blockDim.x) {
            if (a.gout0) a.gout0[size_t(row) * M + q] = double(src[0][q].x);
            if (a.gout1) a.gout1[size_t(row) * M + q] = double(src[0][q].y);
            if (a.gout2) a.gout2[size_t(row) * M + q] = double(src[1][q].x);
        }
        return;
    }

    int nout = 1;
    if (a.mode == RING_RHS) {
        const T fc = T(a.two_omega * a.x[row]);
        for (int q = threadIdx.x; q < M; q += blockDim.x) {
            const T zeta = src[0][q].x, uth = src[0][q].y, uph = src[1][q].x;
            const T qq = zeta + fc;
            src[0][q] = {-qq * uph, qq * uth};
        }
    } else if (a.mode == RING_PROJECT) {
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
        nout = 2;
    }
    __syncthreads();
    stockham<T, TW>(src, dst, nout, plan, tw, -1);

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
        if (nout == 2) {
            // scalar field rho: plain quadrature weight (2 pi / M) w_p
            const T sc2 = scale * T(a.s[row]);
            const cx<T> z = src[1][m];
            ga[(size_t(2) * nlat + row) * ld + m] = {z.x * sc2, z.y * sc2};
        }
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
    a.gsyn = P->d_gsyn;
    a.gana = P->d_gana;
    a.gin0 = gin0;
    a.gin1 = gin1;
    a.gout0 = gout0;
    a.gout1 = gout1;
    a.gout2 = gout2;
    const int nbuf = mode == RING_ADJOINT ? 6 : 4;
    const int threads = P->nlon >= 768 ? 256 : 128;
    if (prec == SPHNSE_FP64) {
        size_t sm = size_t(nbuf) * P->nlon * sizeof(cx<double>);
        cudaFuncSetAttribute(k_ring<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        k_ring<double, double><<<P->nlat, threads, sm, P->stream>>>(a, P->fft, P->d_tw);
    } else {
        size_t sm = size_t(nbuf) * P->nlon * sizeof(cx<float>);
        cudaFuncSetAttribute(k_ring<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        k_ring<float, float><<<P->nlat, threads, sm, P->stream>>>(a, P->fft, P->d_tw32);
    }
    return check_cuda(cudaGetLastError());
}

}  // namespace sph
