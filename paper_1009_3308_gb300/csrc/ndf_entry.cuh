// Per-entry vector operations of the NDF step (Sec. 4.2, Eq. (ode_disc)) on
// one packed entry i of a state with n entries and its backward differences
// D_j (column j at dif + j n), shared by the plan's and the ensemble's kernels.
#pragma once
#include <cuda_runtime.h>

#include "dmath.cuh"
#include "internal.h"
#include "newton.cuh"

namespace sph {

// First differences of a new state: D_0 = h F, D_j = 0 for j >= 1
__device__ __forceinline__ void init_dif_entry(double2* dif, const double2* F, double h, int n, int i) {
    const double2 f = F[i];
    dif[i] = make_double2(h * f.x, h * f.y);
    for (int j = 1; j < SPHNSE_MAXK + 2; ++j) dif[size_t(j) * n + i] = make_double2(0.0, 0.0);
}

// max(|v.x| / max(|y.x|, thr), |v.y| / max(|y.y|, thr)): one entry of the
// weighted max-norm of the initial step (FP64, Newton-refined reciprocals)
__device__ __forceinline__ double wnorm_entry(double2 v, double2 y, double thr) {
    return fmax(fabs(v.x) * rcp64<1>(fmax(fabs(y.x), thr)), fabs(v.y) * rcp64<1>(fmax(fabs(y.y), thr)));
}

// D_j <- sum_l A[l][j] D_l for j < k: the differences re-expressed for a new
// step size (A = R(rho) U, row-major SPHNSE_MAXK x SPHNSE_MAXK)
__device__ __forceinline__ void rescale_entry(double2* dif, const double* A, int k, int n, int i) {
    double2 old[SPHNSE_MAXK];
    for (int j = 0; j < k; ++j) old[j] = dif[size_t(j) * n + i];
    for (int j = 0; j < k; ++j) {
        double sx = 0.0, sy = 0.0;
        for (int l = 0; l < k; ++l) {
            const double a = A[l * SPHNSE_MAXK + j];
            sx += a * old[l].x;
            sy += a * old[l].y;
        }
        dif[size_t(j) * n + i] = make_double2(sx, sy);
    }
}

// Predictor of an attempt of order k: y0 = ynew = y + sum_{j<k} D_j,
// psi = sum_{j<k} g_j D_j, d = 0.  Returns |y| / max(|y|, thr) (FP32, the
// scale of the corrector's rounding-level stop; the max over entries is the
// caller's).
__device__ __forceinline__ float predict_entry(const double2* y, const double2* dif, const double* g, int k,
                                               double2* y0, double2* psi, double2* d, double2* ynew, float thr,
                                               int n, int i) {
    const double2 yi = y[i];
    double2 a = yi, p = make_double2(0.0, 0.0);
    for (int j = 0; j < k; ++j) {
        const double2 dj = dif[size_t(j) * n + i];
        a.x += dj.x;
        a.y += dj.y;
        p.x += g[j] * dj.x;
        p.y += g[j] * dj.y;
    }
    y0[i] = a;
    ynew[i] = a;
    psi[i] = p;
    d[i] = make_double2(0.0, 0.0);
    const float ax = absf_trunc(yi.x), ay = absf_trunc(yi.y);
    return fmaxf(ax / fmaxf(ax, thr), ay / fmaxf(ay, thr));
}

// Accepted step of order k: D_{k+1} = d - D_k; D_k = d; D_j += D_{j+1}
// (j = k-1..0); y = ynew
__device__ __forceinline__ void accept_entry(double2* dif, const double2* d, double2* y, const double2* ynew, int k,
                                             int n, int i) {
    const double2 dd = d[i], dk = dif[size_t(k) * n + i];
    dif[size_t(k + 1) * n + i] = make_double2(dd.x - dk.x, dd.y - dk.y);
    double2 up = dd;
    dif[size_t(k) * n + i] = dd;
    for (int j = k - 1; j >= 0; --j) {
        double2 v = dif[size_t(j) * n + i];
        v.x += up.x;
        v.y += up.y;
        dif[size_t(j) * n + i] = v;
        up = v;
    }
    y[i] = ynew[i];
}

}  // namespace sph
