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

#include "f64cvt.h"

namespace sph {

// The arithmetic is FP32 (the projections are FP32 already): alpha is rounded
// to FP32 and the FP32 result widened exactly, both on the integer ALU, and
// only a nonzero forcing is added in FP64. GB300's FP64 pipe retires about
// two operations per clock per SM, and an FP64 form of this update (14 FP64
// operations per entry) made the finish of a CTA's last order group the tail
// of the fused analysis. The added error (FP32 rounding of nu lam alpha and
// of the Coriolis term, 1e-7 relative) is far below that of the FP32 and
// BF16x3 contractions.
__device__ __forceinline__ double2 finish32_entry(int kind, int L, int m, float4 c, const float* hL, const float* hU,
                                                  const float* hD, double2 a, double2 f, double nu, double omega_d) {
    const float hdr = hD ? hD[2] : 0.f, hdi = hD ? hD[3] : 0.f;
    const float cm = c.x * float(m);
    const float nr = cm * hL[1] - (c.y * hU[2] - c.z * hdr);
    const float ni = -cm * hL[0] - (c.y * hU[3] - c.z * hdi);
    if (kind == 1) return make_double2(f32_to_f64(nr), f32_to_f64(ni));
    (void)L;
    const float ar = f64_to_f32_rn(a.x), ai = f64_to_f32_rn(a.y);
    const float nl = f64_to_f32_rn(nu) * c.w;   // c.w = lam (exact in FP32 for L < 4096)
    float tx = fmaf(-nl, ar, -nr), ty = fmaf(-nl, ai, -ni);
    if (omega_d != 0.0) {
        // 2 Omega m / lam with lam^{-1/2} squared
        const float cor = 2.f * f64_to_f32_rn(omega_d) * float(m) * c.x * c.x;
        tx = fmaf(-cor, ai, tx);
        ty = fmaf(cor, ar, ty);
    }
    double2 r = make_double2(f32_to_f64(tx), f32_to_f64(ty));
    // the forcing's bits decide, not an FP64 compare
    if ((__double_as_longlong(f.x) | __double_as_longlong(f.y)) << 1) {
        r.x += f.x;
        r.y += f.y;
    }
    return r;
}

}  // namespace sph
