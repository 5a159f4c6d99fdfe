// Diagnostics of Sec. 6.2: the energy spectrum E(L) of Eq. (energy), the
// coefficients of a field in the layout of another truncation (P_{N1} of
// Eq. (eq: cut_app_soln) and zero padding), and the approximate inertial
// manifold Phi(u1) = (nu A + C)^{-1} (P_{N2} - P_{N1}) [f - B(u1, u1)] of
// Eq. (eq:p-p), evaluated on a plan of truncation N2 as the RHS at u1 = P_{N1}
// u followed by a diagonal solve on the band N1 < L <= N2 (there u1 and C u1
// vanish, so f - B(u1, u1) = F(u1)).
#include <cuda_runtime.h>

#include "internal.h"

namespace sph {
namespace {

// one warp per degree L: sum over m = 0..L of s_m |alpha_{L,m}|^2 (s_0 = 1,
// s_m = 2: the orders -m), lanes striding over m, then a fixed-order
// butterfly, so the result does not depend on scheduling
__global__ void k_energy(const double2* __restrict__ alpha, double* __restrict__ E, int N) {
    const int L = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (L > N) return;
    double s = 0.0;
    if (L >= 1)
        for (int m = lane; m <= L; m += 32) {
            const double2 a = alpha[packed_index(N, m, L)];
            s += (m == 0 ? 1.0 : 2.0) * (a.x * a.x + a.y * a.y);
        }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) E[L] = s;
}

// out (degree N_out) from in (degree N_in): copy the common modes with
// L <= Lmax, zero the rest
__global__ void k_resize(const double2* __restrict__ in, int N_in, double2* __restrict__ out, int N_out, int Lmax,
                         int n_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_out) return;
    int L, m;
    packed_lm(N_out, i, L, m);
    out[i] = (L <= N_in && L <= Lmax) ? in[packed_index(N_in, m, L)] : make_double2(0.0, 0.0);
}

// phi = F / (nu lambda - 2 i Omega m / lambda) for L > N1, else 0 (in place)
__global__ void k_im_solve(double2* __restrict__ phi, const int2* __restrict__ lm, int N1, double nu, double Omega,
                           int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int L = lm[i].x, m = lm[i].y;
    if (L <= N1) {
        phi[i] = make_double2(0.0, 0.0);
        return;
    }
    const double lam = double(L) * (L + 1.0);
    const double rr = nu * lam, ri = -2.0 * Omega * m / lam;   // (nu A + C) on Z_{L,m}
    const double den = rr * rr + ri * ri;
    const double2 f = phi[i];
    phi[i] = make_double2((f.x * rr + f.y * ri) / den, (f.y * rr - f.x * ri) / den);
}

}  // namespace
}  // namespace sph

using namespace sph;

extern "C" {

int sphnse_energy_spectrum(sphnse_plan* P, const double* alpha, double* E) {
    if (!P || !alpha || !E) return SPHNSE_E_ARG;
    const int wpb = 8;
    k_energy<<<(P->N + wpb) / wpb, 32 * wpb, 0, P->stream>>>(reinterpret_cast<const double2*>(alpha), E, P->N);
    return check_cuda(cudaGetLastError());
}

int sphnse_resize(sphnse_plan* P, int N_in, const double* alpha_in, int L_max, double* alpha_out) {
    if (!P || N_in < 1 || !alpha_in || !alpha_out) return SPHNSE_E_ARG;
    const int n = P->n_coeff;
    k_resize<<<(n + 255) / 256, 256, 0, P->stream>>>(reinterpret_cast<const double2*>(alpha_in), N_in,
                                                     reinterpret_cast<double2*>(alpha_out), P->N,
                                                     L_max < 0 ? P->N : L_max, n);
    return check_cuda(cudaGetLastError());
}

int sphnse_inertial_manifold(sphnse_plan* P, int N1, const double* alpha, const double* forcing, double* phi) {
    if (!P || !alpha || !phi || N1 < 1 || N1 >= P->N || !(P->nu > 0.0)) return SPHNSE_E_ARG;
    const int n = P->n_coeff;
    // u1 = P_{N1} alpha in the plan's step workspace (transient between steps)
    double2* u1 = reinterpret_cast<double2*>(P->d_work);
    k_resize<<<(n + 255) / 256, 256, 0, P->stream>>>(reinterpret_cast<const double2*>(alpha), P->N, u1, P->N, N1, n);
    int rc = check_cuda(cudaGetLastError());
    if (rc) return rc;
    if ((rc = rhs_device(P, reinterpret_cast<const double*>(u1), forcing, phi))) return rc;
    k_im_solve<<<(n + 255) / 256, 256, 0, P->stream>>>(reinterpret_cast<double2*>(phi), P->d_lm, N1, P->nu,
                                                        P->Omega, n);
    return check_cuda(cudaGetLastError());
}

}  // extern "C"
