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

#include "fft_small.cuh"
#include "internal.h"
#include "ptx.cuh"
#include "ring4.cuh"

namespace sph {

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
    allow_dynamic_smem(reinterpret_cast<const void*>(k_ring<T, TW, MODE>), sm);
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
// Four-step ring kernel (the transform itself is in ring4.cuh)

template <int M2>
__global__ void __launch_bounds__(128, 4) k_ring4(Ring4Args a) {
    extern __shared__ __align__(16) float2 sm4[];
    __shared__ float s_rw[128 / M2];
    pdl_launch();
    pdl_wait();
    ring4_rings<M2>(a, blockIdx.x * (128 / M2), blockIdx.y, threadIdx.x, sm4, s_rw, [] { __syncthreads(); });
}

// 256 threads per G = 128 / M2 rings (grids of less than a wave)
template <int M2>
__global__ void __launch_bounds__(256, 3) k_ring4w(Ring4Args a) {
    extern __shared__ __align__(16) float2 sm4[];
    __shared__ float s_rw[128 / M2];
    pdl_launch();
    pdl_wait();
    ring4w_rings<M2>(a, blockIdx.x * (128 / M2), blockIdx.y, threadIdx.x, sm4, s_rw, [] { __syncthreads(); });
}

template <int M2>
static int ring4_t(sphnse_plan* P, int nb, const float* gsyn, size_t sgs, float* gana, size_t sga, int pairs) {
    constexpr size_t sm = ring4_smem<M2>();
    static_assert(sm <= 227 * 1024, "ring4 shared memory");
    allow_dynamic_smem(reinterpret_cast<const void*>(k_ring4<M2>), sm);
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
    const dim3 grid((P->nlat + G - 1) / G, nb);
    if constexpr (M2 >= 16) {
        // a grid of less than four CTAs per SM is latency-bound: twice the
        // threads per ring shorten each thread's chain of passes
        const bool wide = P->ring_threads == 256 ||
                          (P->ring_threads == 0 && size_t(grid.x) * grid.y <= size_t(4) * P->nsm);
        if (wide) {
            allow_dynamic_smem(reinterpret_cast<const void*>(k_ring4w<M2>), sm);
            return check_cuda(launch_pdl(k_ring4w<M2>, grid, dim3(256), sm, P->stream, a));
        }
    }
    return check_cuda(launch_pdl(k_ring4<M2>, grid, dim3(128), sm, P->stream, a));
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
