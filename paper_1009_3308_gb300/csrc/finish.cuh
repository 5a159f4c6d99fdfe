// One packed coefficient of the recombination and diagonal update (A7) on the
// FP32 projections: with the analysis output H of the two product fields at
// the degree-shift rows K = L - 1, L, L + 1 of order m,
//   N_{L,m} = lam^{-1/2} [ -i m H^theta_L - (L eps_{L+1,m} H^phi_{L+1} - (L+1) eps_{L,m} H^phi_{L-1}) ]
// (the transpose of the synthesis' degree-shift recombination), and
//   kind 0: F = fhat - nu lam alpha - N (+ 2 i Omega m / lam alpha with the split Coriolis term),
//   kind 1: the projection N itself.
// c = (lam^{-1/2}, L eps_{L+1,m} lam^{-1/2}, (L+1) eps_{L,m} lam^{-1/2}, lam) in FP32;
// hL, hU, hD: rows of [H^theta re, im, H^phi re, im] (hD null for L - 1 < m).
#pragma once
#include <cuda_runtime.h>

namespace sph {

__device__ __forceinline__ double2 finish32_entry(int kind, int L, int m, float4 c, const float* hL, const float* hU,
                                                  const float* hD, double2 a, double2 f, double nu, double omega_d) {
    const float hdr = hD ? hD[2] : 0.f, hdi = hD ? hD[3] : 0.f;
    const float cm = c.x * float(m);
    const float nr = cm * hL[1] - (c.y * hU[2] - c.z * hdr);
    const float ni = -cm * hL[0] - (c.y * hU[3] - c.z * hdi);
    if (kind == 1) return make_double2(double(nr), double(ni));
    const double nl = nu * (double(L) * double(L + 1));
    double2 r;
    r.x = fma(-nl, a.x, f.x) - double(nr);
    r.y = fma(-nl, a.y, f.y) - double(ni);
    if (omega_d != 0.0) {
        // 2 Omega m / lambda from lambda^{-1/2} in FP32 (relative 1e-7, below
        // the FP32 and BF16x3 paths' own error); FP64 divides are slow here
        const double cor = double(2.f * float(omega_d) * float(m) * c.x * c.x);
        r.x = fma(-cor, a.y, r.x);
        r.y = fma(cor, a.x, r.y);
    }
    return r;
}

}  // namespace sph
