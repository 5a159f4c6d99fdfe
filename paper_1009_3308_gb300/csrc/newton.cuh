// The simplified-Newton update of one packed entry, shared by the plan's and
// the ensemble's corrector kernels (Sec. 4.2, Eq. (ode_disc); the iteration
// matrix is the exact linear part, J_d = -nu lambda_L + 2 i Omega m / lambda_L).
//
// FP64 stays where it decides the result: the residual r = c F - (psi + d),
// the accumulated correction d and the iterate y0 + d, and the differences
// whose norms estimate the error.  What only steers the iteration runs in
// FP32: the iteration matrix 1 / (1 - c J_d) (the iteration converges to the
// FP64 fixed point of the residual whatever its accuracy; a 1e-7 error only
// enters the contraction rate) and the weighted max-norms (2^-23 relative;
// the controller compares them with tolerances).  This part has about 1/64 of
// its FP32 rate in FP64, so the FP64 instruction count is what the kernel's
// time follows.
#pragma once

namespace sph {

// |x| as a float with the top 23 bits of the significand (truncated), from
// integer operations on the two words of the double: exponent rebased from
// 1023 to 127; below the float range 0 or a subnormal, above it FLT_MAX.
// Non-finite inputs give FLT_MAX (see nonfinite_hi).
__device__ __forceinline__ float absf_trunc(double x) {
    const int hi = __double2hiint(x) & 0x7fffffff;
    const unsigned lo = unsigned(__double2loint(x));
    int b = hi - (896 << 20);
    b = min(max(b, 0), 0x0fefffff);
    return __int_as_float((b << 3) | int(lo >> 29));
}

__device__ __forceinline__ bool nonfinite_hi(double x) {
    return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000;
}

struct NewtonEntry {
    double2 dn, yv;   // new correction d and iterate y0 + d
    float nv[4];      // ||dl||, ||d||, ||D_{k-1} + d||, ||d - D_k|| contributions (weighted)
    bool bad;         // a non-finite correction
};

// L, m: degree and order; c = h * iga_k; f = F(ynew); yo = y_n; yn = current
// iterate; dkm1 (nullable) and dk: differences D_{k-1}, D_k
__device__ __forceinline__ NewtonEntry newton_entry(int L, int m, double c, float nu, float two_omega, float thr,
                                                     double2 f, double2 ps, double2 dd, double2 yo, double2 yn,
                                                     double2 a0, const double2* dkm1, double2 dk) {
    NewtonEntry e;
    // 1 / (1 - c J_d), 1 - c J_d = (1 + c nu lam) - i c 2 Omega m / lam, in FP32
    const float lam = float(L * (L + 1));
    const float cf = float(c);
    const float mr = fmaf(cf * nu, lam, 1.f), mi = -cf * two_omega * float(m) / lam;
    const float iden = 1.f / fmaf(mr, mr, mi * mi);
    const double ir = double(mr * iden), ii = double(-mi * iden);
    // FP64: residual, correction, iterate
    const double rx = fma(c, f.x, -(ps.x + dd.x)), ry = fma(c, f.y, -(ps.y + dd.y));
    const double dlx = fma(rx, ir, -ry * ii), dly = fma(ry, ir, rx * ii);
    e.dn = make_double2(dd.x + dlx, dd.y + dly);
    e.yv = make_double2(a0.x + e.dn.x, a0.y + e.dn.y);
    e.bad = nonfinite_hi(dlx) || nonfinite_hi(dly);
    // FP32 weighted norms
    const float ox = absf_trunc(yo.x), oy = absf_trunc(yo.y);
    const float wx = fmaxf(fmaxf(ox, absf_trunc(yn.x)), thr), wy = fmaxf(fmaxf(oy, absf_trunc(yn.y)), thr);
    e.nv[0] = fmaxf(absf_trunc(dlx) / wx, absf_trunc(dly) / wy);
    const float vx = fmaxf(fmaxf(ox, absf_trunc(e.yv.x)), thr), vy = fmaxf(fmaxf(oy, absf_trunc(e.yv.y)), thr);
    const float ivx = 1.f / vx, ivy = 1.f / vy;
    e.nv[1] = fmaxf(absf_trunc(e.dn.x) * ivx, absf_trunc(e.dn.y) * ivy);
    e.nv[2] = 0.f;
    if (dkm1) {
        const double2 q = *dkm1;
        e.nv[2] = fmaxf(absf_trunc(q.x + e.dn.x) * ivx, absf_trunc(q.y + e.dn.y) * ivy);
    }
    e.nv[3] = fmaxf(absf_trunc(e.dn.x - dk.x) * ivx, absf_trunc(e.dn.y - dk.y) * ivy);
    return e;
}

}  // namespace sph
