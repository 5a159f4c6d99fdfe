// Spectral-side kernels of the RHS F (Eq. (ode)) on CUDA cores:
//   prep       coefficient sets for synthesis (Eqs. (stok_eig), (vort_app))
//   synthesis  per-order Legendre sums over the northern nodes, even/odd
//              split (north = E + O, south = E - O)
//   analysis   per-order Legendre sums of the quadrature-weighted Fourier
//              profiles (Eq. (disc_vec_orth_proj))
//   finish     degree-shift recombination and the diagonal Stokes update
//              (Sec. 4.2: nu lambda_L alpha_{L,m}) plus forcing.
// Templated on the contraction type T (double for SPHNSE_FP64, float for
// SPHNSE_FP32); the coefficient state in and out is always FP64.
#include <cuda_runtime.h>

#include "finish.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace sph {

// ---------------------------------------------------------------------------
// prep: one thread per ext row (m, K), K = m..N+1.
//   field 0 (zeta):  lambda_K^{1/2} alpha_K
//   field 1 (theta): a_K = lambda_K^{-1/2} alpha_K
//   field 2 (phi):   (K-1) eps_{K,m} a_{K-1} - (K+2) eps_{K+1,m} a_{K+1}
// (sin(theta) d/dtheta Pt_L^m = L eps_{L+1,m} Pt_{L+1}^m - (L+1) eps_{L,m} Pt_{L-1}^m
//  regrouped by degree).  The FP64 coefficients come precomputed per row
// (c = (lam^{1/2}, lam^{-1/2}, c_down, c_up)) so that the kernel does no
// FP64 square roots or divisions.  With beta (adjoint): fields 3, 4 are the
// theta/phi sets of beta / s_m, s_m = 1 (m = 0) or 2.
template <typename T>
__global__ void k_prep(const double2* __restrict__ alpha, const double2* __restrict__ beta,
                       const double4_32a* __restrict__ prepc, T* __restrict__ bsyn, int N, int nf) {
    // no early trigger: at large L this grid has several waves, and the
    // streaming synthesis after it (programmatic launch, one CTA per SM)
    // would hold SMs its later waves need
    pdl_wait();   // alpha may be the predecessor's output
    const int m = blockIdx.y;
    const int K = m + blockIdx.x * blockDim.x + threadIdx.x;
    if (K > N + 1) return;
    const int lo = m > 0 ? m : 1;
    const int row = ext_row(N, m, K);
    const double4_32a c = prepc[row];
    auto A = [&](const double2* v, int Kp) -> double2 {
        return (Kp < lo || Kp > N) ? make_double2(0.0, 0.0) : v[packed_index(N, m, Kp)];
    };
    T* out = bsyn + size_t(row) * (2 * nf);
    {
        const double2 a0 = A(alpha, K), am = A(alpha, K - 1), ap = A(alpha, K + 1);
        out[0] = T(c.x * a0.x);
        out[1] = T(c.x * a0.y);
        out[2] = T(c.y * a0.x);
        out[3] = T(c.y * a0.y);
        out[4] = T(c.z * am.x + c.w * ap.x);
        out[5] = T(c.z * am.y + c.w * ap.y);
    }
    if (nf == 5) {
        const double sc = m == 0 ? 1.0 : 0.5;
        const double2 b0 = A(beta, K), bm = A(beta, K - 1), bp = A(beta, K + 1);
        out[6] = T(sc * (c.y * b0.x));
        out[7] = T(sc * (c.y * b0.y));
        out[8] = T(sc * (c.z * bm.x + c.w * bp.x));
        out[9] = T(sc * (c.z * bm.y + c.w * bp.y));
    }
}

// FP32-path prep: alpha_K is converted once per row and its degree
// neighbours come from shared memory; the arithmetic is FP32 (the FP32 path
// contracts in FP32 anyway), keeping the weak FP64 pipe for the state only.
__global__ void __launch_bounds__(128) k_prep32(const double2* __restrict__ alpha, const double2* __restrict__ beta,
                                                const float4* __restrict__ prepc, float* __restrict__ bsyn, int N,
                                                int nf, int ncoef, size_t bstride) {
    __shared__ float2 sa[130], sb[130];
    pdl_launch();
    pdl_wait();   // alpha may be the predecessor's output
    // batch of instances along gridDim.z (fixed strides between instances)
    alpha += size_t(blockIdx.z) * ncoef;
    if (beta) beta += size_t(blockIdx.z) * ncoef;
    bsyn += size_t(blockIdx.z) * bstride;
    const int m = blockIdx.y, t = threadIdx.x;
    const int K0 = m + blockIdx.x * 128, K = K0 + t;
    const int lo = m > 0 ? m : 1;
    const float sc = m == 0 ? 1.f : 0.5f;
    auto ld = [&](const double2* v, int Kp, float scale) -> float2 {
        if (Kp < lo || Kp > N) return make_float2(0.f, 0.f);
        const double2 c = v[packed_index(N, m, Kp)];
        return make_float2(float(c.x) * scale, float(c.y) * scale);
    };
    sa[t + 1] = ld(alpha, K, 1.f);
    if (t == 0) sa[0] = ld(alpha, K0 - 1, 1.f);
    if (t == 127) sa[129] = ld(alpha, K0 + 128, 1.f);
    if (nf == 5) {
        sb[t + 1] = ld(beta, K, sc);
        if (t == 0) sb[0] = ld(beta, K0 - 1, sc);
        if (t == 127) sb[129] = ld(beta, K0 + 128, sc);
    }
    __syncthreads();
    if (K > N + 1) return;
    const int row = ext_row(N, m, K);
    const float4 c = prepc[row];
    float* out = bsyn + size_t(row) * (2 * nf);
    const float2 a0 = sa[t + 1], am = sa[t], ap = sa[t + 2];
    out[0] = c.x * a0.x;
    out[1] = c.x * a0.y;
    out[2] = c.y * a0.x;
    out[3] = c.y * a0.y;
    out[4] = fmaf(c.z, am.x, c.w * ap.x);
    out[5] = fmaf(c.z, am.y, c.w * ap.y);
    if (nf == 5) {
        const float2 b0 = sb[t + 1], bm = sb[t], bp = sb[t + 2];
        out[6] = c.y * b0.x;
        out[7] = c.y * b0.y;
        out[8] = fmaf(c.z, bm.x, c.w * bp.x);
        out[9] = fmaf(c.z, bm.y, c.w * bp.y);
    }
}

// ---------------------------------------------------------------------------
// synthesis: block (p-tile, m); thread = one northern node p.
//   g_f(theta_p) = sum_K Pt_K^m(x_p) b_{f,K}: even rows E, odd rows O;
//   north row p: E + O, south row nlat-1-p: E - O.
// Field scalings: theta fields (i m / sin), phi fields (-1 / sin), zeta none.
// Output gsyn[f][row][m] complex.
template <typename T, int NF>
__global__ void __launch_bounds__(128) k_synthesis(const T* __restrict__ psyn, const T* __restrict__ bsyn,
                                                    T* __restrict__ gsyn, const double* __restrict__ sinth,
                                                    int N, int nh, int nlat, int pairs) {
    pdl_launch();
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* B = reinterpret_cast<T*>(smem_raw);
    const int m = blockIdx.y;
    const int e0 = ext_off(N, m), cnt = ext_count(N, m), ne = ext_even(N, m), no = ext_odd(N, m);
    for (int i = threadIdx.x; i < cnt * 2 * NF; i += blockDim.x) B[i] = bsyn[size_t(e0) * 2 * NF + i];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nh) return;
    T ev[2 * NF], od[2 * NF];
#pragma unroll
    for (int f = 0; f < 2 * NF; ++f) { ev[f] = T(0); od[f] = T(0); }
    const T* Pe = psyn + size_t(e0) * nh + p;
#pragma unroll 4
    for (int j = 0; j < ne; ++j) {
        const T pv = __ldg(Pe + size_t(j) * nh);
        const T* b = B + j * 2 * NF;
#pragma unroll
        for (int f = 0; f < 2 * NF; ++f) ev[f] = fma(pv, b[f], ev[f]);
    }
    const T* Po = psyn + size_t(e0 + ne) * nh + p;
#pragma unroll 4
    for (int j = 0; j < no; ++j) {
        const T pv = __ldg(Po + size_t(j) * nh);
        const T* b = B + (ne + j) * 2 * NF;
#pragma unroll
        for (int f = 0; f < 2 * NF; ++f) od[f] = fma(pv, b[f], od[f]);
    }
    const T inv_s = T(1.0 / sinth[p]);
    const T mm = T(m);
#pragma unroll
    for (int hemi = 0; hemi < 2; ++hemi) {
        const int row = hemi == 0 ? p : nlat - 1 - p;
        if (hemi == 1 && row == p) break;  // equator of an odd grid
        const T sg = hemi == 0 ? T(1) : T(-1);
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            T gr = ev[2 * f] + sg * od[2 * f];
            T gi = ev[2 * f + 1] + sg * od[2 * f + 1];
            T outr, outi;
            if (f == 0) {
                outr = gr; outi = gi;
            } else if (f == 1 || f == 3) {  // (i m / sin) g
                outr = -mm * gi * inv_s;
                outi = mm * gr * inv_s;
            } else {                         // -(1 / sin) g
                outr = -gr * inv_s;
                outi = -gi * inv_s;
            }
            T* dst = gsyn + gsyn_index(pairs, f, m, row, N, nlat) * 2;
            dst[0] = outr;
            dst[1] = outi;
        }
    }
}

// ---------------------------------------------------------------------------
// analysis: block (j-tile, m, parity); thread = one ext row (degree K).
//   H_{f,K} = sum_{north p} Pt_K^m(x_p) [G_f(p) + (-1)^{K+m} G_f(p')],
// p' the mirror row; the table block is [nh][rows] so that threads of a warp
// read consecutive degrees.  G already carries (2 pi / M) w_p / sin(theta_p)
// (and sin(theta_p) for the scalar adjoint field).
template <typename T, int NF>
__global__ void __launch_bounds__(128) k_analysis(const T* __restrict__ pana, const T* __restrict__ gana,
                                                   T* __restrict__ hana, int N, int nh, int nlat) {
    pdl_launch();
    pdl_wait();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);  // [nh][2 NF]
    const int m = blockIdx.y, par = blockIdx.z;
    const int ne = ext_even(N, m), no = ext_odd(N, m);
    const int nrows = par ? no : ne;
    if (int(blockIdx.x * blockDim.x) >= nrows) return;
    const int rowstart = ext_off(N, m) + (par ? ne : 0);
    const size_t ld = size_t(N + 1);
    for (int i = threadIdx.x; i < nh * NF; i += blockDim.x) {
        const int p = i / NF, f = i % NF;
        const int pr = nlat - 1 - p;
        const T* a = gana + ((size_t(f) * ld + m) * nlat + p) * 2;
        T ar = a[0], ai = a[1], br = T(0), bi = T(0);
        if (pr != p) {
            const T* b = gana + ((size_t(f) * ld + m) * nlat + pr) * 2;
            br = b[0];
            bi = b[1];
        }
        S[p * 2 * NF + 2 * f] = par ? ar - br : ar + br;
        S[p * 2 * NF + 2 * f + 1] = par ? ai - bi : ai + bi;
    }
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nrows) return;
    T acc[2 * NF];
#pragma unroll
    for (int f = 0; f < 2 * NF; ++f) acc[f] = T(0);
    const T* Pa = pana + size_t(rowstart) * nh + j;
#pragma unroll 4
    for (int p = 0; p < nh; ++p) {
        const T pv = __ldg(Pa + size_t(p) * nrows);
        const T* sp = S + p * 2 * NF;
#pragma unroll
        for (int f = 0; f < 2 * NF; ++f) acc[f] = fma(pv, sp[f], acc[f]);
    }
    T* dst = hana + size_t(rowstart + j) * 2 * NF;
#pragma unroll
    for (int f = 0; f < 2 * NF; ++f) dst[f] = acc[f];
}

// ---------------------------------------------------------------------------
// finish: one thread per packed (L, m).
//   N_{L,m} = lambda^{-1/2} [ -i m H^theta_L
//             - (L eps_{L+1,m} H^phi_{L+1} - (L+1) eps_{L,m} H^phi_{L-1}) ]
// with the FP64 coefficients precomputed per entry:
// c = (lambda^{-1/2}, L eps_{L+1,m} lambda^{-1/2}, (L+1) eps_{L,m} lambda^{-1/2}, lambda).
// kind 0: out = forcing - nu lambda alpha - N              (Eq. (ode));
//         + 2 i omega_d m / lambda alpha, the Coriolis diagonal of
//         Eq. (Coriolis_ZLm), when the product leaves it out (omega_d = Omega)
// kind 1: out = N                                          (projection)
// kind 2: out = -nu lambda w - s_m (N + lambda^{1/2} H^rho_L)  (J^T w; alpha = w)
template <typename T>
__global__ void k_finish(int kind, const T* __restrict__ hana, int nf, const double2* __restrict__ alpha,
                         const double2* __restrict__ forcing, double2* __restrict__ out,
                         const int2* __restrict__ lm, const double4_32a* __restrict__ finc, int N, double nu,
                         int n, double omega_d) {
    pdl_launch();
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int L = lm[i].x, m = lm[i].y;
    const double4_32a c = finc[i];
    const T* hL = hana + size_t(ext_row(N, m, L)) * 2 * nf;
    const T* hU = hana + size_t(ext_row(N, m, L + 1)) * 2 * nf;
    const double htr = double(hL[0]), hti = double(hL[1]);
    const double hur = double(hU[2]), hui = double(hU[3]);
    double hdr = 0.0, hdi = 0.0;
    if (L - 1 >= m) {
        const T* hD = hana + size_t(ext_row(N, m, L - 1)) * 2 * nf;
        hdr = double(hD[2]);
        hdi = double(hD[3]);
    }
    const double cm = c.x * m;
    const double nr = cm * hti - (c.y * hur - c.z * hdr);
    const double ni = -cm * htr - (c.y * hui - c.z * hdi);
    const double lam = c.w;
    double2 r;
    if (kind == 0) {
        const double2 a = alpha[i];
        const double2 f = forcing ? forcing[i] : make_double2(0.0, 0.0);
        r.x = f.x - nu * lam * a.x - nr;
        r.y = f.y - nu * lam * a.y - ni;
        if (omega_d != 0.0) {
            const double cor = 2.0 * omega_d * m / lam;
            r.x -= cor * a.y;
            r.y += cor * a.x;
        }
    } else if (kind == 1) {
        r = make_double2(nr, ni);
    } else {
        const double2 wv = alpha[i];
        const double sm = m == 0 ? 1.0 : 2.0;
        const double sl = lam * c.x;  // lambda^{1/2}
        r.x = -nu * lam * wv.x - sm * (nr + sl * double(hL[4]));
        r.y = -nu * lam * wv.y - sm * (ni + sl * double(hL[5]));
    }
    out[i] = r;
}

// FP32-path finish: the recombination runs in FP32 on the FP32 projections
// (coefficients in FP32); only the state update f - nu lambda alpha - N is
// FP64.
__global__ void k_finish32(int kind, const float* __restrict__ hana, int nf, const double2* __restrict__ alpha,
                           const double2* __restrict__ forcing, double2* __restrict__ out,
                           const int2* __restrict__ lm, const float4* __restrict__ finc, int N, double nu, int n,
                           size_t hstride, const double* __restrict__ nu_inst, double omega_d) {
    pdl_launch();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // the plan's constants are read before the wait for the predecessor
    int L, m;
    packed_lm(N, i, L, m);
    (void)lm;
    const float4 c = finc[i];
    pdl_wait();
    // batch of instances along gridDim.y: per-instance vectors, projections, nu
    {
        const size_t b = blockIdx.y;
        hana += b * hstride;
        alpha += b * n;
        out += b * n;
        if (forcing) forcing += b * n;
        if (nu_inst) nu = nu_inst[b];
    }
    const float* hL = hana + size_t(ext_row(N, m, L)) * 2 * nf;
    const float* hU = hana + size_t(ext_row(N, m, L + 1)) * 2 * nf;
    const float* hD = L - 1 >= m ? hana + size_t(ext_row(N, m, L - 1)) * 2 * nf : nullptr;
    double2 r;
    if (kind < 2) {
        const double2 a = kind == 0 ? alpha[i] : make_double2(0.0, 0.0);
        const double2 f = kind == 0 && forcing ? forcing[i] : make_double2(0.0, 0.0);
        r = finish32_entry(kind, L, m, c, hL, hU, hD, a, f, nu, omega_d);
    } else {
        const float hdr = hD ? hD[2] : 0.f, hdi = hD ? hD[3] : 0.f;
        const float cm = c.x * float(m);
        const float nr = cm * hL[1] - (c.y * hU[2] - c.z * hdr);
        const float ni = -cm * hL[0] - (c.y * hU[3] - c.z * hdi);
        const double lam = double(L) * double(L + 1);
        const double2 wv = alpha[i];
        const float sm = m == 0 ? 1.f : 2.f;
        const float sl = c.w * c.x;  // lambda^{1/2}
        const double nl = nu * lam;
        r.x = -nl * wv.x - double(sm * (nr + sl * hL[4]));
        r.y = -nl * wv.y - double(sm * (ni + sl * hL[5]));
    }
    out[i] = r;
}

// ---------------------------------------------------------------------------
// launchers

template <typename T>
static int prep_t(sphnse_plan* P, const double* alpha, const double* beta) {
    const int nf = beta ? 5 : 3;
    dim3 blk(128), grd((P->N + 2 + 127) / 128, P->N + 1);
    stage_begin(P, SPHNSE_STAGE_PREP);
    launch_pdl_small(P->n_cta, k_prep<T>, grd, blk, 0, P->stream, reinterpret_cast<const double2*>(alpha),
               reinterpret_cast<const double2*>(beta), static_cast<const double4_32a*>(P->d_prepc),
               reinterpret_cast<T*>(P->d_bsyn), P->N, nf);
    stage_end(P, SPHNSE_STAGE_PREP);
    return check_cuda(cudaGetLastError());
}

int launch_prep(sphnse_plan* P, const double* alpha, const double* beta, int prec) {
    if (prec == SPHNSE_FP64) return prep_t<double>(P, alpha, beta);
    const int nf = beta ? 5 : 3;
    dim3 blk(128), grd((P->N + 2 + 127) / 128, P->N + 1);
    stage_begin(P, SPHNSE_STAGE_PREP);
    launch_pdl(k_prep32, grd, blk, 0, P->stream, reinterpret_cast<const double2*>(alpha),
               reinterpret_cast<const double2*>(beta), static_cast<const float4*>(P->d_prepc32),
               reinterpret_cast<float*>(P->d_bsyn), P->N, nf, P->n_coeff, size_t(0));
    stage_end(P, SPHNSE_STAGE_PREP);
    return check_cuda(cudaGetLastError());
}

template <typename T, int NF>
static int synth_t(sphnse_plan* P, int pairs) {
    dim3 blk(128), grd((P->nh + 127) / 128, P->N + 1);
    size_t sm = size_t(P->N + 2) * 2 * NF * sizeof(T);
    if (sm > 48 * 1024)
        allow_dynamic_smem(reinterpret_cast<const void*>(k_synthesis<T, NF>), sm);
    stage_begin(P, SPHNSE_STAGE_SYNTHESIS);
    launch_pdl_small(P->n_cta, k_synthesis<T, NF>, grd, blk, sm, P->stream,
               reinterpret_cast<const T*>(P->tab[sizeof(T) == 8 ? SPHNSE_FP64 : SPHNSE_FP32].syn),
               reinterpret_cast<const T*>(P->d_bsyn), reinterpret_cast<T*>(P->d_gsyn),
               static_cast<const double*>(P->d_s), P->N, P->nh, P->nlat, pairs);
    stage_end(P, SPHNSE_STAGE_SYNTHESIS);
    return check_cuda(cudaGetLastError());
}

int launch_synthesis(sphnse_plan* P, int nfields, int prec, int pairs) {
    if (stream_ok(P, prec)) {
        int rc = launch_synthesis_stream(P, nfields, prec, pairs);
        if (rc != SPHNSE_E_UNSUPPORTED) return rc;
    }
    if (prec == SPHNSE_FP64) return nfields == 5 ? synth_t<double, 5>(P, pairs) : synth_t<double, 3>(P, pairs);
    return nfields == 5 ? synth_t<float, 5>(P, pairs) : synth_t<float, 3>(P, pairs);
}

template <typename T, int NF>
static int anal_t(sphnse_plan* P) {
    const int maxrows = ext_even(P->N, 0);
    dim3 blk(128), grd((maxrows + 127) / 128, P->N + 1, 2);
    size_t sm = size_t(P->nh) * 2 * NF * sizeof(T);
    if (sm > 48 * 1024) {
        allow_dynamic_smem(reinterpret_cast<const void*>(k_analysis<T, NF>), sm);
    }
    stage_begin(P, SPHNSE_STAGE_ANALYSIS);
    launch_pdl_small(P->n_cta, k_analysis<T, NF>, grd, blk, sm, P->stream,
               reinterpret_cast<const T*>(P->tab[sizeof(T) == 8 ? SPHNSE_FP64 : SPHNSE_FP32].ana),
               reinterpret_cast<const T*>(P->d_gana), reinterpret_cast<T*>(P->d_hana), P->N, P->nh, P->nlat);
    stage_end(P, SPHNSE_STAGE_ANALYSIS);
    return check_cuda(cudaGetLastError());
}

int launch_analysis(sphnse_plan* P, int nfields, int prec) {
    if (stream_ok(P, prec)) {
        int rc = launch_analysis_stream(P, nfields, prec);
        if (rc != SPHNSE_E_UNSUPPORTED) return rc;
    }
    if (prec == SPHNSE_FP64) return nfields == 3 ? anal_t<double, 3>(P) : anal_t<double, 2>(P);
    return nfields == 3 ? anal_t<float, 3>(P) : anal_t<float, 2>(P);
}

int launch_finish(sphnse_plan* P, int kind, int prec, const double* alpha, const double* forcing,
                  double* out) {
    const int n = P->n_coeff;
    const int nf = kind == 2 ? 3 : 2;
    dim3 blk(256), grd((n + 255) / 256);
    stage_begin(P, SPHNSE_STAGE_FINISH);
    if (prec == SPHNSE_FP64)
        launch_pdl_small(P->n_cta, k_finish<double>, grd, blk, 0, P->stream, kind, static_cast<const double*>(P->d_hana), nf,
                                                     reinterpret_cast<const double2*>(alpha),
                                                     reinterpret_cast<const double2*>(forcing),
                                                     reinterpret_cast<double2*>(out), P->d_lm, P->d_finc, P->N, P->nu, n,
                                                     kind == 0 && P->coriolis_split ? P->Omega : 0.0);
    else
        launch_pdl(k_finish32, grd, blk, 0, P->stream, kind, static_cast<const float*>(P->d_hana), nf,
                   reinterpret_cast<const double2*>(alpha), reinterpret_cast<const double2*>(forcing),
                   reinterpret_cast<double2*>(out), static_cast<const int2*>(P->d_lm),
                   static_cast<const float4*>(P->d_finc32), P->N, P->nu, n, size_t(0),
                   static_cast<const double*>(nullptr), kind == 0 && P->coriolis_split ? P->Omega : 0.0);
    stage_end(P, SPHNSE_STAGE_FINISH);
    return check_cuda(cudaGetLastError());
}

// batched FP32 launchers over nb instances with fixed strides (ensemble)
int launch_prep32_batch(sphnse_plan* P, int nb, const double* alpha, float* bsyn, size_t bstride) {
    dim3 blk(128), grd((P->N + 2 + 127) / 128, P->N + 1, nb);
    stage_begin(P, SPHNSE_STAGE_PREP);
    launch_pdl(k_prep32, grd, blk, 0, P->stream, reinterpret_cast<const double2*>(alpha),
               static_cast<const double2*>(nullptr), static_cast<const float4*>(P->d_prepc32), bsyn, P->N, 3,
               P->n_coeff, bstride);
    stage_end(P, SPHNSE_STAGE_PREP);
    return check_cuda(cudaGetLastError());
}

int launch_finish32_batch(sphnse_plan* P, int nb, const float* hana, size_t hstride, const double* alpha,
                          double* out, const double* nu_inst) {
    const int n = P->n_coeff;
    dim3 blk(256), grd((n + 255) / 256, nb);
    stage_begin(P, SPHNSE_STAGE_FINISH);
    launch_pdl(k_finish32, grd, blk, 0, P->stream, 0, hana, 2, reinterpret_cast<const double2*>(alpha),
               static_cast<const double2*>(nullptr), reinterpret_cast<double2*>(out),
               static_cast<const int2*>(P->d_lm), static_cast<const float4*>(P->d_finc32), P->N, P->nu, n, hstride,
               nu_inst, 0.0);
    stage_end(P, SPHNSE_STAGE_FINISH);
    return check_cuda(cudaGetLastError());
}

}  // namespace sph
