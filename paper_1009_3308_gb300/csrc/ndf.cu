// Variable-order, variable-step NDF integrator (Sec. 4.2, Eq. (ode_disc)),
// its frozen-controller replay, and the discrete adjoint of that replay.
//
// The controller (host) follows the quasi-constant step-size NDF scheme of
// the MATLAB ODE suite that the paper cites: backward differences D_j =
// nabla^{j+1} alpha_n, predictor alpha0 = alpha_n + sum_{j<k} D_j, corrector
//   c F(t_{n+1}, alpha0 + d) - psi - d = 0,  c = h / ((1 - kappa_k) gamma_k),
//   psi = sum_{j<k} gamma_{j+1} D_j / ((1 - kappa_k) gamma_k),
// solved by simplified Newton with the diagonal iteration matrix
// I - c J_d, J_d = -nu lambda_L + 2 i Omega m / lambda_L (the exact linear
// part, Eq. (Coriolis_ZLm) and the Stokes eigenvalues); error estimate
// (kappa_k gamma_k + 1/(k+1)) ||d / wt||_inf, wt = max(|alpha_n|,
// |alpha_{n+1}|, atol/rtol) per real component; order and step selection from
// the estimates of orders k-1, k, k+1; difference rescaling by R(rho) U on a
// step-size change.  All vector work is FP64 on the device; the host reads
// four norms per Newton iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "dmath.cuh"
#include "newton.cuh"
#include "reduce.cuh"

namespace sph {

namespace {

const double KAPPA[SPHNSE_MAXK] = {-0.1850, -1.0 / 9.0, -0.0823, -0.0415, 0.0};

struct NDFConst {
    double kappa[SPHNSE_MAXK], gamma[SPHNSE_MAXK], iga[SPHNSE_MAXK], ec[SPHNSE_MAXK];
    explicit NDFConst(bool bdf) {
        double g = 0.0;
        for (int k = 1; k <= SPHNSE_MAXK; ++k) {
            g += 1.0 / k;
            kappa[k - 1] = bdf ? 0.0 : KAPPA[k - 1];
            gamma[k - 1] = g;
            iga[k - 1] = 1.0 / (g * (1.0 - kappa[k - 1]));
            ec[k - 1] = kappa[k - 1] * g + 1.0 / (k + 1.0);
        }
    }
};

struct Mat { double a[SPHNSE_MAXK * SPHNSE_MAXK]; };
struct Coef { double c[SPHNSE_MAXK]; };

// (R(rho) U)[:k, :k], R_ij = prod_{l=1..i} (l - 1 - j rho) / l, U = R(1)
Mat rescale_matrix(int k, double rho) {
    double R[SPHNSE_MAXK][SPHNSE_MAXK], U[SPHNSE_MAXK][SPHNSE_MAXK];
    for (int j = 1; j <= k; ++j) {
        double r = 1.0, u = 1.0;
        for (int i = 1; i <= k; ++i) {
            r *= (i - 1.0 - j * rho) / i;
            u *= (i - 1.0 - j) / i;
            R[i - 1][j - 1] = r;
            U[i - 1][j - 1] = u;
        }
    }
    Mat m;
    std::memset(&m, 0, sizeof(m));
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += R[i][l] * U[l][j];
            m.a[i * SPHNSE_MAXK + j] = s;
        }
    return m;
}

inline double d2u_max(unsigned long long v) {
    double d;
    std::memcpy(&d, &v, sizeof(d));
    return d;
}

}  // namespace

// ---------------------------------------------------------------------------
// device kernels (one thread per packed complex entry)


__global__ void k_zero_dif(double2* dif, const double2* F, double h, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 f = F[i];
    dif[i] = make_double2(h * f.x, h * f.y);
    for (int j = 1; j < SPHNSE_MAXK + 2; ++j) dif[size_t(j) * n + i] = make_double2(0.0, 0.0);
}

// ||v / max(|y|, thr)||_inf into slot
__global__ void k_wnorm(const double2* v, const double2* y, double thr, unsigned long long* slots, int idx, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double r[1] = {0.0};
    if (i < n) {
        const double2 a = v[i], b = y[i];
        r[0] = fmax(fabs(a.x) * rcp64<1>(fmax(fabs(b.x), thr)), fabs(a.y) * rcp64<1>(fmax(fabs(b.y), thr)));
    }
    const int id[1] = {idx};
    block_amax<1>(slots, r, id);
}

__global__ void k_rescale(double2* dif, Mat A, int k, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 old[SPHNSE_MAXK];
    for (int j = 0; j < k; ++j) old[j] = dif[size_t(j) * n + i];
    for (int j = 0; j < k; ++j) {
        double sx = 0.0, sy = 0.0;
        for (int l = 0; l < k; ++l) {
            const double a = A.a[l * SPHNSE_MAXK + j];
            sx += a * old[l].x;
            sy += a * old[l].y;
        }
        dif[size_t(j) * n + i] = make_double2(sx, sy);
    }
}

// y0 = y + sum_{j<k} D_j,  psi = sum_{j<k} g_j D_j,  d = 0,  ynew = y0
// and slot 4 = ||y / max(|y|, thr)||_inf, the scale of the corrector's
// rounding-level stop (FP32, like the corrector's other norms)
__global__ void k_predict(const double2* y, const double2* dif, Coef g, int k, double2* y0, double2* psi,
                          double2* d, double2* ynew, float thr, unsigned long long* slots, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float r[1] = {0.f};
    if (i < n) {
        const double2 yi = y[i];
        double2 a = yi, p = make_double2(0.0, 0.0);
        for (int j = 0; j < k; ++j) {
            const double2 dj = dif[size_t(j) * n + i];
            a.x += dj.x;
            a.y += dj.y;
            p.x += g.c[j] * dj.x;
            p.y += g.c[j] * dj.y;
        }
        y0[i] = a;
        ynew[i] = a;
        psi[i] = p;
        d[i] = make_double2(0.0, 0.0);
        const float ax = absf_trunc(yi.x), ay = absf_trunc(yi.y);
        r[0] = fmaxf(ax / fmaxf(ax, thr), ay / fmaxf(ay, thr));
    }
    const int id[1] = {4};
    block_amax_f<1>(slots, r, id, false);
}

// One simplified-Newton update: r = c F - (psi + d), dl = r / (1 - c J_d),
// d += dl, ynew = y0 + d, and the four weighted max-norms:
// slot0 ||dl||  (weights from the pre-update ynew), slot1 ||d||,
// slot2 ||D_{k-1} + d||, slot3 ||d - D_k||  (weights from the new ynew).
__global__ void k_newton(const double2* F, const double2* y, const double2* y0, const double2* psi, double2* d,
                         double2* ynew, const double2* dkm1, const double2* dk, const int2* lm, double c,
                         double nu, double Omega, double thr, unsigned long long* slot, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float nv[4] = {0.f, 0.f, 0.f, 0.f};
    bool bad = false;
    if (i < n) {
        const int2 q = lm[i];
        const NewtonEntry e = newton_entry(q.x, q.y, c, float(nu), float(2.0 * Omega), fmaxf(float(thr), 1e-30f),
                                           F[i], psi[i], d[i], y[i], ynew[i], y0[i], dkm1 ? dkm1 + i : nullptr, dk[i]);
        d[i] = e.dn;
        ynew[i] = e.yv;
        for (int j = 0; j < 4; ++j) nv[j] = e.nv[j];
        bad = e.bad;
    }
    const int id[4] = {0, 1, 2, 3};
    block_amax_f<4>(slot, nv, id, bad);
}

// The same update with its parameters read from the device-side loop state
// (a graph node keeps fixed arguments; c, k and the weights change per attempt)
__global__ void k_newton_g(const double2* F, const double2* y, const double2* y0, const double2* psi, double2* d,
                           double2* ynew, const double2* dif, const int2* lm, const NewtonCtl* ctl,
                           unsigned long long* slot, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = ctl->k;
    float nv[4] = {0.f, 0.f, 0.f, 0.f};
    bool bad = false;
    if (i < n) {
        const int2 q = lm[i];
        const NewtonEntry e = newton_entry(q.x, q.y, ctl->c, float(ctl->nu), float(2.0 * ctl->omega),
                                           fmaxf(float(ctl->thr), 1e-30f), F[i], psi[i], d[i], y[i], ynew[i], y0[i],
                                           k >= 2 ? dif + size_t(k - 1) * n + i : nullptr, dif[size_t(k) * n + i]);
        d[i] = e.dn;
        ynew[i] = e.yv;
        for (int j = 0; j < 4; ++j) nv[j] = e.nv[j];
        bad = e.bad;
    }
    const int id[4] = {0, 1, 2, 3};
    block_amax_f<4>(slot, nv, id, bad);
}

// One thread: the corrector's stopping rule after iteration ctl->it (the same
// tests as the host loop), then clear the slots the next iteration fills and
// set the WHILE condition (0: stop).
__global__ void k_newton_ctl(NewtonCtl* ctl, unsigned long long* slots, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double eps = 2.220446049250313e-16;
    const int it = ctl->it;
    bool stop = false, conv = false;
    if (slots[7]) {
        ctl->nonfinite = 1;
        stop = true;
    } else {
        double nv[4];
        for (int q = 0; q < 4; ++q) nv[q] = __longlong_as_double(static_cast<long long>(slots[q]));
        if (it == 0) ctl->ynorm = __longlong_as_double(static_cast<long long>(slots[4]));
        ctl->its = it + 1;
        for (int q = 0; q < 4; ++q) ctl->nrm[q] = nv[q];
        const double newnrm = nv[0], minnrm = 100.0 * eps * ctl->ynorm, oldnrm = ctl->oldnrm;
        const double rtol = ctl->rtol;
        if (ctl->tight) {
            const bool stalled = !ctl->fp64 && it >= 3 && newnrm > 0.8 * oldnrm;
            if (newnrm <= fmax(minnrm, 1e-15) || stalled) stop = conv = true;
        } else if (newnrm <= minnrm) {
            stop = conv = true;
        } else if (it == 0) {
            if (ctl->havrate) {
                const double errit = newnrm * ctl->rate / (1.0 - ctl->rate);
                if (errit <= 0.05 * rtol) stop = conv = true;
            } else {
                ctl->rate = 0.0;
            }
        } else if (newnrm > 0.9 * oldnrm) {
            stop = true;   // too slow
        } else {
            ctl->rate = fmax(0.9 * ctl->rate, newnrm / oldnrm);
            ctl->havrate = 1;
            const double errit = newnrm * ctl->rate / (1.0 - ctl->rate);
            if (errit <= 0.5 * rtol) stop = conv = true;
            else if (it == ctl->maxit - 1) stop = true;
            else if (0.5 * rtol < errit * pow(ctl->rate, double(ctl->maxit - 1 - it))) stop = true;
        }
        ctl->oldnrm = newnrm;
        if (!stop && it + 1 >= ctl->maxit) {
            stop = true;
            conv = ctl->tight != 0;   // the host loop: a tight loop that ran out counts as converged
        }
    }
    ctl->it = it + 1;
    ctl->conv = conv;
    ctl->stop = stop;
    for (int q = 0; q < 4; ++q) slots[q] = 0ull;
    slots[7] = 0ull;
    cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// D_{k+1} = d - D_k; D_k = d; D_j += D_{j+1} (j = k-1..0); y = ynew
__global__ void k_accept(double2* dif, const double2* d, double2* y, const double2* ynew, int k, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
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

// ---------------------------------------------------------------------------
// adjoint kernels

// reverse of k_accept: G = dbar (in place), abar = adjoint of ynew.
// dbar'_j (j < k) = sum_{i<=j} G_i;  dbar_k = -G_{k+1};  dbar_{k+1} = 0;
// dtot = sum_{i<=k} G_i + G_{k+1} + abar (adjoint of d); y0bar = abar.
__global__ void k_adj_accept(double2* dbar, const double2* abar, double2* dtot, int k, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 cum = make_double2(0.0, 0.0);
    for (int j = 0; j < k; ++j) {
        const double2 g = dbar[size_t(j) * n + i];
        cum.x += g.x;
        cum.y += g.y;
        dbar[size_t(j) * n + i] = cum;
    }
    const double2 gk = dbar[size_t(k) * n + i], gk1 = dbar[size_t(k + 1) * n + i], a = abar[i];
    dtot[i] = make_double2(cum.x + gk.x + gk1.x + a.x, cum.y + gk.y + gk1.y + a.y);
    dbar[size_t(k) * n + i] = make_double2(-gk1.x, -gk1.y);
    dbar[size_t(k + 1) * n + i] = make_double2(0.0, 0.0);
}

// mu <- mu + (b - mu + c JT) / conj(1 - c J_d); slot0 = ||b - mu + c JT||_inf (abs)
__global__ void k_adj_fixpoint(double2* mu, const double2* b, const double2* JT, const int2* lm, double c,
                               double nu, double Omega, unsigned long long* slot, int first, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double r[1] = {0.0};
    if (i < n) {
        const int L = lm[i].x, m = lm[i].y;
        const double lam = double(L) * (L + 1.0);
        const double mr = 1.0 + c * nu * lam, mi = c * 2.0 * Omega * m * rcp64<2>(lam);  // conj(1 - c J_d)
        const double2 bb = b[i];
        double rx, ry;
        double2 u = make_double2(0.0, 0.0);
        if (first) {
            rx = bb.x;
            ry = bb.y;
        } else {
            u = mu[i];
            const double2 jt = JT[i];
            rx = bb.x - u.x + c * jt.x;
            ry = bb.y - u.y + c * jt.y;
        }
        r[0] = fmax(fabs(rx), fabs(ry));
        const double iden = rcp64<2>(mr * mr + mi * mi);
        u.x += (rx * mr + ry * mi) * iden;
        u.y += (ry * mr - rx * mi) * iden;
        mu[i] = u;
    }
    const int id[1] = {0};
    block_amax<1>(slot, r, id);
}

// y0bar = abar + mu - dtot;  dbar_j += g_j (-mu) + y0bar (j < k);  abar = y0bar;
// partial sums of <lambda ynew, mu> for the nu gradient
__global__ void k_adj_finish(double2* abar, double2* dbar, const double2* mu, const double2* dtot,
                             const double2* ynew, const int2* lm, Coef g, int k, double* part, int n) {
    __shared__ double red[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n) {
        const double2 u = mu[i], a = abar[i], dt = dtot[i];
        const double2 y0b = make_double2(a.x + u.x - dt.x, a.y + u.y - dt.y);
        for (int j = 0; j < k; ++j) {
            double2 v = dbar[size_t(j) * n + i];
            v.x += -g.c[j] * u.x + y0b.x;
            v.y += -g.c[j] * u.y + y0b.y;
            dbar[size_t(j) * n + i] = v;
        }
        abar[i] = y0b;
        const int L = lm[i].x;
        const double lam = double(L) * (L + 1.0);
        const double2 yn = ynew[i];
        s = lam * (yn.x * u.x + yn.y * u.y);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// dbar_i (i < k) = sum_j A_ij dbar'_j
__global__ void k_adj_rescale(double2* dbar, Mat A, int k, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 v[SPHNSE_MAXK];
    for (int j = 0; j < k; ++j) v[j] = dbar[size_t(j) * n + i];
    for (int r = 0; r < k; ++r) {
        double sx = 0.0, sy = 0.0;
        for (int j = 0; j < k; ++j) {
            const double a = A.a[r * SPHNSE_MAXK + j];
            sx += a * v[j].x;
            sy += a * v[j].y;
        }
        dbar[size_t(r) * n + i] = make_double2(sx, sy);
    }
}

// out += s * v (complex, real scalar s)
__global__ void k_axpy(double2* out, const double2* v, double s, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 o = out[i];
    const double2 a = v[i];
    o.x += s * a.x;
    o.y += s * a.y;
    out[i] = o;
}

// partial sums of <lambda alpha, w>
__global__ void k_lam_dot(const double2* alpha, const double2* w, const int2* lm, double* part, int n) {
    __shared__ double red[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n) {
        const int L = lm[i].x;
        const double2 a = alpha[i], b = w[i];
        s = double(L) * (L + 1.0) * (a.x * b.x + a.y * b.y);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int wd = 128; wd > 0; wd >>= 1) {
        if (threadIdx.x < wd) red[threadIdx.x] += red[threadIdx.x + wd];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// objective: rows outside [theta_lo, theta_hi] are zeroed in place; per row
// the partial (2 pi / M) w_p / 2 sum_q |u|^2 of the band rows
__global__ void k_band(double* uth, double* uph, const double* theta, const double* w, double lo, double hi,
                       int M, double* part) {
    __shared__ double red[256];
    const int row = blockIdx.x;
    const bool in = theta[row] >= lo && theta[row] <= hi;
    double s = 0.0;
    for (int q = threadIdx.x; q < M; q += blockDim.x) {
        const size_t o = size_t(row) * M + q;
        if (in) s += uth[o] * uth[o] + uph[o] * uph[o];
        else uth[o] = uph[o] = 0.0;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int wd = 128; wd > 0; wd >>= 1) {
        if (threadIdx.x < wd) red[threadIdx.x] += red[threadIdx.x + wd];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[row] = in ? 0.5 * (2.0 * 3.14159265358979323846 / M) * w[row] * red[0] : 0.0;
}

// grad = s_m (proj + 2 (alpha - target)); partial sums of s_m |alpha - target|^2
__global__ void k_obj_grad(const double2* alpha, const double2* tgt, const double2* proj, double2* grad,
                           const int2* lm, double* part, int n) {
    __shared__ double red[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n) {
        const double sm = lm[i].y == 0 ? 1.0 : 2.0;
        const double2 a = alpha[i], t = tgt ? tgt[i] : make_double2(0.0, 0.0), p = proj[i];
        const double dx = a.x - t.x, dy = a.y - t.y;
        grad[i] = make_double2(sm * (p.x + 2.0 * dx), sm * (p.y + 2.0 * dy));
        s = sm * (dx * dx + dy * dy);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int wd = 128; wd > 0; wd >>= 1) {
        if (threadIdx.x < wd) red[threadIdx.x] += red[threadIdx.x + wd];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------
// host helpers

namespace {

struct Work {
    double2 *y0, *psi, *d, *ynew, *F, *mu, *dtot, *jt;
    double* part;  // block partial sums
};

Work work(sphnse_plan* P) {
    const size_t n = P->n_coeff;
    double2* w = reinterpret_cast<double2*>(P->d_work);
    Work r;
    r.y0 = w;
    r.psi = w + n;
    r.d = w + 2 * n;
    r.ynew = w + 3 * n;
    r.F = w + 4 * n;
    r.mu = w + 5 * n;
    r.dtot = w + 6 * n;
    r.jt = w + 7 * n;
    r.part = reinterpret_cast<double*>(w + 8 * n);
    return r;
}

inline dim3 grid(int n) { return dim3((n + 255) / 256); }

// the eight norm slots through the plan's pinned mirror (a pageable
// destination would be staged by the driver)
int read_norms(sphnse_plan* P, double* out, int cnt) {
    unsigned long long* h = reinterpret_cast<unsigned long long*>(P->h_norms);
    if (cudaMemcpyAsync(h, P->d_norms, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, P->stream) !=
        cudaSuccess)
        return SPHNSE_E_CUDA;
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return SPHNSE_E_CUDA;
    if (h[7]) return SPHNSE_E_NONFINITE;
    for (int i = 0; i < cnt; ++i) out[i] = d2u_max(h[i]);
    return SPHNSE_OK;
}

int clear_norms(sphnse_plan* P) {
    return cudaMemsetAsync(P->d_norms, 0, 8 * sizeof(unsigned long long), P->stream) == cudaSuccess
               ? SPHNSE_OK
               : SPHNSE_E_CUDA;
}

double sum_partials(sphnse_plan* P, const double* part, int nblk, int* rc) {
    std::vector<double> h(nblk);
    if (cudaMemcpyAsync(h.data(), part, nblk * sizeof(double), cudaMemcpyDeviceToHost, P->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess) {
        *rc = SPHNSE_E_CUDA;
        return 0.0;
    }
    double s = 0.0;
    for (double v : h) s += v;  // fixed order: deterministic
    return s;
}

int stage_launch_check(sphnse_plan* P) { return check_cuda(cudaGetLastError()); }

// rescale the first k differences from h_dif to h (no-op when equal)
int rescale(sphnse_plan* P, sphnse_state* st, double h, int k) {
    if (h == st->h_dif) return SPHNSE_OK;
    const Mat A = rescale_matrix(k, h / st->h_dif);
    stage_begin(P, SPHNSE_STAGE_STEP);
    k_rescale<<<grid(P->n_coeff), 256, 0, P->stream>>>(reinterpret_cast<double2*>(st->dif), A, k, P->n_coeff);
    stage_end(P, SPHNSE_STAGE_STEP);
    st->h_dif = h;
    st->nconhk = 0;
    return stage_launch_check(P);
}

// The corrector's Newton loop as one graph launch: a WHILE node whose body is
// the RHS at ynew, the Newton update and the control kernel, which sets the
// loop condition on the device, so an attempt costs one host round trip
// instead of one per iteration.  Built per (state, forcing, precision, nu,
// Omega) after the plan's kernels are set up; any failure to capture leaves
// the host loop in charge.
bool newton_graph_ready(sphnse_plan* P, sphnse_state* st, const double* forcing) {
    if (P->ng_failed || P->timing) return false;
    const void* key[4] = {st->alpha, st->dif, forcing,
                          reinterpret_cast<const void*>(uintptr_t(P->precision) | (uintptr_t(P->coriolis_split) << 8))};
    if (P->ng_exec && std::equal(key, key + 4, P->ng_key) && P->ng_nu == P->nu && P->ng_omega == P->Omega) return true;
    if (P->ng_exec) {
        cudaGraphExecDestroy(P->ng_exec);
        P->ng_exec = nullptr;
    }
    if (!P->d_ctl && (cudaMalloc(reinterpret_cast<void**>(&P->d_ctl), sizeof(NewtonCtl)) != cudaSuccess ||
                      cudaMallocHost(reinterpret_cast<void**>(&P->h_ctl), sizeof(NewtonCtl)) != cudaSuccess)) {
        P->ng_failed = true;
        return false;
    }
    if (!P->cap_stream && cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        P->ng_failed = true;
        return false;
    }
    // the body's kernels must not set anything up while being captured
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return false;
    Work W = work(P);
    const int n = P->n_coeff;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (ok) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        const cudaStream_t saved = P->stream;
        P->stream = P->cap_stream;
        ok = cudaStreamBeginCaptureToGraph(P->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) ==
             cudaSuccess;
        if (ok) {
            const int rc = rhs_device(P, reinterpret_cast<const double*>(W.ynew), forcing,
                                      reinterpret_cast<double*>(W.F));
            k_newton_g<<<grid(n), 256, 0, P->cap_stream>>>(
                W.F, reinterpret_cast<const double2*>(st->alpha), W.y0, W.psi, W.d, W.ynew,
                reinterpret_cast<const double2*>(st->dif), P->d_lm, P->d_ctl, P->d_norms, n);
            k_newton_ctl<<<1, 32, 0, P->cap_stream>>>(P->d_ctl, P->d_norms, h);
            cudaGraph_t out = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(P->cap_stream, &out);
            ok = rc == SPHNSE_OK && ce == cudaSuccess;
        }
        P->stream = saved;
    }
    if (ok) ok = cudaGraphInstantiate(&P->ng_exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();   // a failed capture leaves no sticky error; clear the last one
    if (!ok) {
        P->ng_exec = nullptr;
        P->ng_failed = true;
        return false;
    }
    std::copy(key, key + 4, P->ng_key);
    P->ng_nu = P->nu;
    P->ng_omega = P->Omega;
    return true;
}

// Predictor + simplified Newton.  tight: iterate until the update norm is
// below max(minnrm, 1e-15) (replay).  Returns SPHNSE_OK / error; *conv set.
int corrector(sphnse_plan* P, sphnse_state* st, const double* forcing, double h, int k, bool tight, int maxit,
              const NDFConst& C, bool* conv, int* its, double norms[4]) {
    const int n = P->n_coeff;
    Work W = work(P);
    const double thr = P->atol / P->rtol;
    if (h != st->miter_h || k != st->miter_k) {
        st->havrate = 0;
        st->miter_h = h;
        st->miter_k = k;
    }
    Coef g;
    for (int j = 0; j < SPHNSE_MAXK; ++j) g.c[j] = j < k ? C.gamma[j] * C.iga[k - 1] : 0.0;
    int rc;
    if ((rc = clear_norms(P))) return rc;
    stage_begin(P, SPHNSE_STAGE_STEP);
    k_predict<<<grid(n), 256, 0, P->stream>>>(reinterpret_cast<const double2*>(st->alpha),
                                               reinterpret_cast<const double2*>(st->dif), g, k, W.y0, W.psi, W.d,
                                               W.ynew, fmaxf(float(thr), 1e-30f), P->d_norms, n);
    stage_end(P, SPHNSE_STAGE_STEP);
    if ((rc = stage_launch_check(P))) return rc;
    const double cc = h * C.iga[k - 1];
    if (newton_graph_ready(P, st, forcing)) {
        NewtonCtl& q = *P->h_ctl;
        std::memset(&q, 0, sizeof(q));
        q.c = cc;
        q.nu = P->nu;
        q.omega = P->Omega;
        q.thr = thr;
        q.rtol = P->rtol;
        q.rate = st->rate;
        q.havrate = st->havrate;
        q.k = k;
        q.maxit = maxit;
        q.tight = tight;
        q.fp64 = P->precision == SPHNSE_FP64;
        if (cudaMemcpyAsync(P->d_ctl, P->h_ctl, sizeof(NewtonCtl), cudaMemcpyHostToDevice, P->stream) != cudaSuccess ||
            cudaGraphLaunch(P->ng_exec, P->stream) != cudaSuccess ||
            cudaMemcpyAsync(P->h_ctl, P->d_ctl, sizeof(NewtonCtl), cudaMemcpyDeviceToHost, P->stream) != cudaSuccess ||
            cudaStreamSynchronize(P->stream) != cudaSuccess)
            return SPHNSE_E_CUDA;
        if (q.nonfinite) return SPHNSE_E_NONFINITE;
        *conv = q.conv != 0;
        *its = q.its;
        for (int j = 0; j < 4; ++j) norms[j] = q.nrm[j];
        st->rate = q.rate;
        st->havrate = q.havrate;
        return SPHNSE_OK;
    }
    const double eps = 2.220446049250313e-16;
    double oldnrm = 0.0, ynorm = 0.0;
    *conv = false;
    for (int it = 0; it < maxit; ++it) {
        if ((rc = rhs_device(P, reinterpret_cast<const double*>(W.ynew), forcing,
                             reinterpret_cast<double*>(W.F))))
            return rc;
        if (it > 0 && (rc = clear_norms(P))) return rc;
        stage_begin(P, SPHNSE_STAGE_STEP);
        k_newton<<<grid(n), 256, 0, P->stream>>>(
            W.F, reinterpret_cast<const double2*>(st->alpha), W.y0, W.psi, W.d, W.ynew,
            k >= 2 ? reinterpret_cast<const double2*>(st->dif) + size_t(k - 1) * n : nullptr,
            reinterpret_cast<const double2*>(st->dif) + size_t(k) * n, P->d_lm, cc, P->nu, P->Omega, thr,
            P->d_norms, n);
        stage_end(P, SPHNSE_STAGE_STEP);
        if ((rc = stage_launch_check(P))) return rc;
        double nv[5];
        if ((rc = read_norms(P, nv, it == 0 ? 5 : 4))) return rc;
        if (it == 0) ynorm = nv[4];
        *its = it + 1;
        for (int q = 0; q < 4; ++q) norms[q] = nv[q];
        const double newnrm = nv[0];
        const double minnrm = 100.0 * eps * ynorm;
        if (tight) {
            // converged to the rounding level: below 1e-15 in the weighted
            // norm, or no longer shrinking (FP32 / BF16 contractions stall at
            // their own rounding level long before 1e-15)
            const bool stalled = P->precision != SPHNSE_FP64 && it >= 3 && newnrm > 0.8 * oldnrm;
            if (newnrm <= std::max(minnrm, 1e-15) || stalled) {
                *conv = true;
                return SPHNSE_OK;
            }
            oldnrm = newnrm;
            continue;
        }
        if (newnrm <= minnrm) {
            *conv = true;
            return SPHNSE_OK;
        }
        if (it == 0) {
            if (st->havrate) {
                const double errit = newnrm * st->rate / (1.0 - st->rate);
                if (errit <= 0.05 * P->rtol) {
                    *conv = true;
                    return SPHNSE_OK;
                }
            } else {
                st->rate = 0.0;
            }
        } else if (newnrm > 0.9 * oldnrm) {
            return SPHNSE_OK;  // too slow
        } else {
            st->rate = std::max(0.9 * st->rate, newnrm / oldnrm);
            st->havrate = 1;
            const double errit = newnrm * st->rate / (1.0 - st->rate);
            if (errit <= 0.5 * P->rtol) {
                *conv = true;
                return SPHNSE_OK;
            }
            if (it == maxit - 1) return SPHNSE_OK;
            if (0.5 * P->rtol < errit * std::pow(st->rate, maxit - 1 - it)) return SPHNSE_OK;
        }
        oldnrm = newnrm;
    }
    if (tight) *conv = true;
    return SPHNSE_OK;
}

int accept(sphnse_plan* P, sphnse_state* st, int k) {
    Work W = work(P);
    stage_begin(P, SPHNSE_STAGE_STEP);
    k_accept<<<grid(P->n_coeff), 256, 0, P->stream>>>(reinterpret_cast<double2*>(st->dif), W.d,
                                                      reinterpret_cast<double2*>(st->alpha), W.ynew, k,
                                                      P->n_coeff);
    stage_end(P, SPHNSE_STAGE_STEP);
    return stage_launch_check(P);
}

}  // namespace
}  // namespace sph

using namespace sph;

extern "C" {

int sphnse_state_init(sphnse_plan* P, sphnse_state* st, double t0, double h0, const double* forcing) {
    if (!P || !st || !st->alpha || !st->dif || !std::isfinite(t0)) return SPHNSE_E_ARG;
    const int n = P->n_coeff;
    Work W = work(P);
    int rc;
    if ((rc = rhs_device(P, st->alpha, forcing, reinterpret_cast<double*>(W.F)))) return rc;
    if (!(h0 > 0.0)) {
        const double thr = P->atol / P->rtol;
        if ((rc = clear_norms(P))) return rc;
        k_wnorm<<<grid(n), 256, 0, P->stream>>>(W.F, reinterpret_cast<const double2*>(st->alpha), thr,
                                                 P->d_norms, 0, n);
        double nv[1];
        if ((rc = read_norms(P, nv, 1))) return rc;
        const double rh = 1.25 * nv[0] / std::sqrt(P->rtol);
        h0 = rh > 0.0 ? std::min(P->h_max, 1.0 / rh) : P->h_max;
    }
    k_zero_dif<<<grid(n), 256, 0, P->stream>>>(reinterpret_cast<double2*>(st->dif), W.F, h0, n);
    if ((rc = check_cuda(cudaGetLastError()))) return rc;
    st->t = t0;
    st->h = h0;
    st->order = 1;
    st->h_dif = h0;
    st->nconhk = 0;
    st->havrate = 0;
    st->rate = 0.0;
    st->miter_h = 0.0;
    st->miter_k = 0;
    if (!(st->t_end > t0)) st->t_end = INFINITY;
    return SPHNSE_OK;
}

int sphnse_step(sphnse_plan* P, sphnse_state* st, const double* forcing, sphnse_step_info* info) {
    if (!P || !st || !st->alpha || !st->dif) return SPHNSE_E_ARG;
    const NDFConst C(P->bdf != 0);
    const int maxk = P->max_order;
    bool nofailed = true;
    int rejections = 0, newton_total = 0, rhs_evals = 0;
    const double h_dif_before = st->h_dif;
    const double eps16 = 16.0 * 2.220446049250313e-16;
    int rc;
    for (int attempt = 0; attempt < 200; ++attempt) {
        const double hmin = eps16 * std::fabs(st->t);
        double h = std::min(P->h_max, std::max(hmin, st->h));
        if (1.1 * h >= st->t_end - st->t) h = st->t_end - st->t;
        st->h = h;
        int k = st->order;
        if ((rc = rescale(P, st, h, k))) return rc;
        bool conv;
        int its = 0;
        double nrm[4];
        if ((rc = corrector(P, st, forcing, h, k, false, P->newton_max, C, &conv, &its, nrm))) return rc;
        newton_total += its;
        rhs_evals += its;
        if (!conv) {
            ++rejections;
            if (h <= hmin) return SPHNSE_E_STEP_TOO_SMALL;
            st->h = std::max(hmin, 0.3 * h);
            continue;
        }
        const double err = nrm[1] * C.ec[k - 1];
        if (err > P->rtol) {
            ++rejections;
            if (h <= hmin) return SPHNSE_E_STEP_TOO_SMALL;
            if (nofailed) {
                nofailed = false;
                double hopt = h * std::max(0.1, 0.833 * std::pow(P->rtol / err, 1.0 / (k + 1)));
                if (k > 1) {
                    const double errkm1 = nrm[2] * C.ec[k - 2];
                    const double hkm1 = h * std::max(0.1, 0.769 * std::pow(P->rtol / errkm1, 1.0 / k));
                    if (hkm1 > hopt) {
                        hopt = std::min(h, hkm1);
                        st->order = k - 1;
                    }
                }
                st->h = std::max(hmin, hopt);
            } else {
                st->h = std::max(hmin, 0.5 * h);
            }
            continue;
        }
        // accepted
        if ((rc = accept(P, st, k))) return rc;
        st->t += h;
        st->nconhk = std::min(st->nconhk + 1, SPHNSE_MAXK + 2);
        if (st->nconhk >= k + 2) {
            double temp = 1.2 * std::pow(err / P->rtol, 1.0 / (k + 1));
            double hopt = temp > 0.1 ? h / temp : 10.0 * h;
            int kopt = k;
            if (k > 1) {
                const double errkm1 = nrm[2] * C.ec[k - 2];
                temp = 1.3 * std::pow(errkm1 / P->rtol, 1.0 / k);
                const double hkm1 = temp > 0.1 ? h / temp : 10.0 * h;
                if (hkm1 > hopt) {
                    hopt = hkm1;
                    kopt = k - 1;
                }
            }
            if (k < maxk) {
                const double errkp1 = nrm[3] * C.ec[k];
                temp = 1.4 * std::pow(errkp1 / P->rtol, 1.0 / (k + 2));
                const double hkp1 = temp > 0.1 ? h / temp : 10.0 * h;
                if (hkp1 > hopt) {
                    hopt = hkp1;
                    kopt = k + 1;
                }
            }
            if (hopt > h) {
                st->h = hopt;
                if (kopt != k) {
                    st->order = kopt;
                    st->nconhk = 0;
                }
            }
        }
        if (info) {
            info->t = st->t;
            info->h = h;
            info->err = err;
            info->order = k;
            info->newton_iters = newton_total;
            info->rejections = rejections;
            info->rhs_evals = rhs_evals;
            info->next_order = st->order;
            info->next_h = st->h;
            info->h_dif_before = h_dif_before;
        }
        return SPHNSE_OK;
    }
    return SPHNSE_E_STEP_TOO_SMALL;
}

int sphnse_advance(sphnse_plan* P, sphnse_state* st, const double* forcing, int nsteps, sphnse_step_info* info) {
    if (!P || !st || nsteps < 0) return SPHNSE_E_ARG;
    for (int s = 0; s < nsteps; ++s) {
        const int rc = sphnse_step(P, st, forcing, info ? info + s : nullptr);
        if (rc) return rc;
    }
    return SPHNSE_OK;
}

int sphnse_replay_step(sphnse_plan* P, sphnse_state* st, const double* forcing, double h, int k, int newton_max,
                       sphnse_step_info* info) {
    if (!P || !st || !(h > 0.0) || k < 1 || k > SPHNSE_MAXK || newton_max < 1) return SPHNSE_E_ARG;
    const NDFConst C(P->bdf != 0);
    const double h_dif_before = st->h_dif;
    st->order = k;
    int rc;
    if ((rc = rescale(P, st, h, k))) return rc;
    bool conv;
    int its = 0;
    double nrm[4];
    if ((rc = corrector(P, st, forcing, h, k, true, newton_max, C, &conv, &its, nrm))) return rc;
    if ((rc = accept(P, st, k))) return rc;
    st->t += h;
    st->h = h;
    if (info) {
        info->t = st->t;
        info->h = h;
        info->err = nrm[1] * C.ec[k - 1];
        info->order = k;
        info->newton_iters = its;
        info->rejections = 0;
        info->rhs_evals = its;
        info->next_order = k;
        info->next_h = h;
        info->h_dif_before = h_dif_before;
    }
    return SPHNSE_OK;
}

int sphnse_rhs_adjoint(sphnse_plan* P, const double* alpha, const double* w, double* out, double* nu_bar) {
    if (!P || !alpha || !w || !out || out == w) return SPHNSE_E_ARG;
    int rc;
    if ((rc = rhs_adjoint_device(P, alpha, w, out))) return rc;
    if (nu_bar) {
        Work W = work(P);
        const int n = P->n_coeff, nb = (n + 255) / 256;
        k_lam_dot<<<nb, 256, 0, P->stream>>>(reinterpret_cast<const double2*>(alpha),
                                             reinterpret_cast<const double2*>(w), P->d_lm, W.part, n);
        *nu_bar -= sum_partials(P, W.part, nb, &rc);
    }
    return rc;
}

int sphnse_adjoint_init(sphnse_plan* P, double h0, const double* alpha0, double* abar, const double* dbar,
                        double* nu_bar) {
    if (!P || !alpha0 || !abar || !dbar) return SPHNSE_E_ARG;
    Work W = work(P);
    const int n = P->n_coeff;
    int rc;
    // D_0 = h0 F(alpha0): abar += h0 J^T dbar_0, nu_bar += h0 <dbar_0, -lambda alpha0>
    if ((rc = rhs_adjoint_device(P, alpha0, dbar, reinterpret_cast<double*>(W.jt)))) return rc;
    k_axpy<<<grid(n), 256, 0, P->stream>>>(reinterpret_cast<double2*>(abar), W.jt, h0, n);
    if (nu_bar) {
        const int nb = (n + 255) / 256;
        k_lam_dot<<<nb, 256, 0, P->stream>>>(reinterpret_cast<const double2*>(alpha0),
                                             reinterpret_cast<const double2*>(dbar), P->d_lm, W.part, n);
        *nu_bar -= h0 * sum_partials(P, W.part, nb, &rc);
    }
    return rc ? rc : check_cuda(cudaGetLastError());
}

int sphnse_adjoint_step(sphnse_plan* P, double h, int k, double h_dif_before, const double* alpha_next,
                        double* abar, double* dbar, double* nu_bar) {
    if (!P || !(h > 0.0) || k < 1 || k > SPHNSE_MAXK || !alpha_next || !abar || !dbar) return SPHNSE_E_ARG;
    const NDFConst C(P->bdf != 0);
    const int n = P->n_coeff;
    Work W = work(P);
    double2* ab = reinterpret_cast<double2*>(abar);
    double2* db = reinterpret_cast<double2*>(dbar);
    int rc;
    stage_begin(P, SPHNSE_STAGE_STEP);
    k_adj_accept<<<grid(n), 256, 0, P->stream>>>(db, ab, W.dtot, k, n);
    stage_end(P, SPHNSE_STAGE_STEP);
    // (I - c J^T) mu = dtot by preconditioned fixed-point iteration
    const double c = h * C.iga[k - 1];
    double scale = -1.0, prev = 0.0;
    for (int it = 0; it < 200; ++it) {
        if (it > 0 && (rc = rhs_adjoint_device(P, alpha_next, reinterpret_cast<const double*>(W.mu),
                                               reinterpret_cast<double*>(W.jt))))
            return rc;
        if ((rc = clear_norms(P))) return rc;
        stage_begin(P, SPHNSE_STAGE_STEP);
        k_adj_fixpoint<<<grid(n), 256, 0, P->stream>>>(W.mu, W.dtot, W.jt, P->d_lm, c, P->nu, P->Omega,
                                                       P->d_norms, it == 0, n);
        stage_end(P, SPHNSE_STAGE_STEP);
        double r[1];
        if ((rc = read_norms(P, r, 1))) return rc;
        if (it == 0) scale = r[0];
        // converged, or stalled at the rounding level of the contractions
        const bool stalled = P->precision != SPHNSE_FP64 && it >= 3 && r[0] > 0.8 * prev;
        if (r[0] <= 1e-14 * scale || scale == 0.0 || stalled) break;
        prev = r[0];
    }
    Coef g;
    for (int j = 0; j < SPHNSE_MAXK; ++j) g.c[j] = j < k ? C.gamma[j] * C.iga[k - 1] : 0.0;
    const int nb = (n + 255) / 256;
    stage_begin(P, SPHNSE_STAGE_STEP);
    k_adj_finish<<<nb, 256, 0, P->stream>>>(ab, db, W.mu, W.dtot, reinterpret_cast<const double2*>(alpha_next),
                                            P->d_lm, g, k, W.part, n);
    stage_end(P, SPHNSE_STAGE_STEP);
    // nu_bar += c <F_nu(ynew), mu> = -c <lambda ynew, mu>
    const double dot = sum_partials(P, W.part, nb, &rc);
    if (rc) return rc;
    if (nu_bar) *nu_bar -= c * dot;
    if (h != h_dif_before) {
        const Mat A = rescale_matrix(k, h / h_dif_before);
        stage_begin(P, SPHNSE_STAGE_STEP);
        k_adj_rescale<<<grid(n), 256, 0, P->stream>>>(db, A, k, n);
        stage_end(P, SPHNSE_STAGE_STEP);
    }
    return check_cuda(cudaGetLastError());
}

int sphnse_objective(sphnse_plan* P, const double* alpha, const double* target, double theta_lo,
                     double theta_hi, double* J, double* grad) {
    if (!P || !alpha || !J || !grad) return SPHNSE_E_ARG;
    const int n = P->n_coeff;
    const size_t gsz = size_t(P->nlat) * P->nlon;
    if (!P->d_grid) {
        if (cudaMalloc(reinterpret_cast<void**>(&P->d_grid), 2 * gsz * sizeof(double)) != cudaSuccess)
            return SPHNSE_E_NOMEM;
        if (cudaMalloc(reinterpret_cast<void**>(&P->d_theta), P->nlat * sizeof(double)) != cudaSuccess)
            return SPHNSE_E_NOMEM;
        if (cudaMalloc(reinterpret_cast<void**>(&P->d_w), P->nlat * sizeof(double)) != cudaSuccess)
            return SPHNSE_E_NOMEM;
        cudaMemcpy(P->d_theta, P->theta.data(), P->nlat * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(P->d_w, P->w.data(), P->nlat * sizeof(double), cudaMemcpyHostToDevice);
    }
    double* uth = P->d_grid;
    double* uph = P->d_grid + gsz;
    Work W = work(P);
    int rc;
    if ((rc = sphnse_grid_fields(P, alpha, nullptr, uth, uph))) return rc;
    k_band<<<P->nlat, 256, 0, P->stream>>>(uth, uph, P->d_theta, P->d_w, theta_lo, theta_hi, P->nlon, W.part);
    if ((rc = check_cuda(cudaGetLastError()))) return rc;
    const double ke = sum_partials(P, W.part, P->nlat, &rc);
    if (rc) return rc;
    if ((rc = sphnse_project(P, uth, uph, reinterpret_cast<double*>(W.jt)))) return rc;
    const int nb = (n + 255) / 256;
    k_obj_grad<<<nb, 256, 0, P->stream>>>(reinterpret_cast<const double2*>(alpha),
                                          reinterpret_cast<const double2*>(target), W.jt,
                                          reinterpret_cast<double2*>(grad), P->d_lm, W.part, n);
    const double mis = sum_partials(P, W.part, nb, &rc);
    *J = ke + mis;
    return rc ? rc : check_cuda(cudaGetLastError());
}

}  // extern "C"
