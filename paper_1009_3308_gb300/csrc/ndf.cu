// Variable-order, variable-step NDF integrator (Sec. 4.2, Eq. (ode_disc)),
// its frozen-controller replay, and the discrete adjoint of that replay.
//
// The controller follows the quasi-constant step-size NDF scheme of
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
// step-size change.  All vector work is FP64 on the device.  The controller
// (att_begin / att_end, newton_control) runs on the device inside one graph
// launch per call (nested WHILE nodes over attempts and Newton iterations),
// or on the host with the same functions when stage timing is on.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "controller.cuh"
#include "dmath.cuh"
#include "ndf_entry.cuh"
#include "newton.cuh"
#include "reduce.cuh"

namespace sph {

namespace {

struct NDFConst {
    double gamma[SPHNSE_MAXK], iga[SPHNSE_MAXK], ec[SPHNSE_MAXK];
    explicit NDFConst(bool bdf) { ndf_constants(bdf, gamma, iga, ec); }
};

struct Mat { double a[SPHNSE_MAXK * SPHNSE_MAXK]; };
struct Coef { double c[SPHNSE_MAXK]; };

Mat rescale_matrix(int k, double rho) {
    Mat m;
    rescale_matrix_into(k, rho, m.a);
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
    if (i < n) init_dif_entry(dif, F, h, n, i);
}

// ||v / max(|y|, thr)||_inf into slot
__global__ void k_wnorm(const double2* v, const double2* y, double thr, unsigned long long* slots, int idx, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double r[1] = {0.0};
    if (i < n) r[0] = wnorm_entry(v[i], y[i], thr);
    const int id[1] = {idx};
    block_amax<1>(slots, r, id);
}

__global__ void k_rescale(double2* dif, Mat A, int k, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rescale_entry(dif, A.a, k, n, i);
}

// y0 = y + sum_{j<k} D_j,  psi = sum_{j<k} g_j D_j,  d = 0,  ynew = y0
// and slot 4 = ||y / max(|y|, thr)||_inf, the scale of the corrector's
// rounding-level stop (FP32, like the corrector's other norms)
__device__ __forceinline__ void predict_block(const double2* y, const double2* dif, const double* g, int k,
                                              double2* y0, double2* psi, double2* d, double2* ynew, float thr,
                                              unsigned long long* slots, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float r[1] = {0.f};
    if (i < n) r[0] = predict_entry(y, dif, g, k, y0, psi, d, ynew, thr, n, i);
    const int id[1] = {4};
    block_amax_f<1>(slots, r, id, false);
}

__global__ void k_predict(const double2* y, const double2* dif, Coef g, int k, double2* y0, double2* psi,
                          double2* d, double2* ynew, float thr, unsigned long long* slots, int n) {
    predict_block(y, dif, g.c, k, y0, psi, d, ynew, thr, slots, n);
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

// The same update inside the graphs' Newton loop: parameters read from the
// device-side loop state (a graph node keeps fixed arguments; c, k and the
// weights change per attempt), and the last block to finish applies the
// stopping rule to the iteration's norms, clears the slots the next
// iteration fills and sets the WHILE condition (0: stop).
__global__ void k_newton_g(const double2* F, const double2* y, const double2* y0, const double2* psi, double2* d,
                           double2* ynew, const double2* dif, const int2* lm, NewtonCtl* ctl,
                           unsigned long long* slot, int n, cudaGraphConditionalHandle h) {
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
    __threadfence();   // this block's slot updates before its arrival
    __syncthreads();
    if (threadIdx.x != 0 || atomicAdd(&ctl->arrived, 1u) != gridDim.x - 1) return;
    __threadfence();
    double v[5];
    for (int q = 0; q < 5; ++q) v[q] = __longlong_as_double(static_cast<long long>(__ldcg(slot + q)));
    const bool stop = newton_control(*ctl, v, __ldcg(slot + 7) != 0ull);
    for (int q = 0; q < 4; ++q) slot[q] = 0ull;
    slot[7] = 0ull;
    ctl->arrived = 0u;
    cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// D_{k+1} = d - D_k; D_k = d; D_j += D_{j+1} (j = k-1..0); y = ynew
__global__ void k_accept(double2* dif, const double2* d, double2* y, const double2* ynew, int k, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) accept_entry(dif, d, y, ynew, k, n, i);
}

// The step loop's kernels.  Per attempt: k_prepare (the previous attempt's
// accept if it was accepted, the rescale to this attempt's h, the predictor;
// all three per entry), the Newton loop, k_step_next (one thread).  The loop
// is entered through k_step_begin and left through k_accept_g.

// one thread: the first attempt's parameters; clear the norm slots
__global__ void k_step_begin(StepCtl* S, unsigned long long* slots) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    att_begin(*S);
    for (int q = 0; q < 8; ++q) slots[q] = 0ull;
}

__global__ void k_prepare(double2* y, double2* dif, double2* y0, double2* psi, double2* d, double2* ynew,
                          const StepCtl* S, unsigned long long* slots, cudaGraphConditionalHandle newton, int n) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(newton, 1u);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        if (S->accept) accept_entry(dif, d, y, ynew, S->k_acc, n, i);
        if (S->do_rescale) rescale_entry(dif, S->A, S->k, n, i);
    }
    predict_block(y, dif, S->g, S->k, y0, psi, d, ynew, fmaxf(float(S->thr), 1e-30f), slots, n);
}

// one thread: finish the attempt, start the next one if the loop goes on
__global__ void k_step_next(StepCtl* S, unsigned long long* slots, cudaGraphConditionalHandle loop) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    att_end(*S);
    const bool more = S->status == SPHNSE_OK && S->done < S->nsteps;
    if (more) att_begin(*S);
    for (int q = 0; q < 8; ++q) slots[q] = 0ull;
    cudaGraphSetConditional(loop, more ? 1u : 0u);
}

// the last attempt's accept, after the loop
__global__ void k_accept_g(double2* dif, const double2* d, double2* y, const double2* ynew, const StepCtl* S, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && S->accept) accept_entry(dif, d, y, ynew, S->k_acc, n, i);
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

// the five slots a Newton iteration reads, and whether a non-finite value was seen
int read_newton_norms(sphnse_plan* P, double* nv, bool* bad) {
    unsigned long long* h = reinterpret_cast<unsigned long long*>(P->h_norms);
    if (cudaMemcpyAsync(h, P->d_norms, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, P->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess)
        return SPHNSE_E_CUDA;
    *bad = h[7] != 0ull;
    for (int i = 0; i < 5; ++i) nv[i] = d2u_max(h[i]);
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

int stage_launch_check(sphnse_plan*) { return check_cuda(cudaGetLastError()); }

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
// the RHS at ynew and the Newton update, whose last block sets the loop
// condition on the device, so an attempt costs one host round trip
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
                reinterpret_cast<const double2*>(st->dif), P->d_lm, P->d_ctl, P->d_norms, n, h);
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

// Predictor (weights g) + simplified Newton with the parameters in q; the
// results (convergence, iterations, norms, rate memory) come back in q.  The
// iterations run as one graph launch when the Newton graph is available, else
// one by one from the host with the same stopping rule.
int corrector(sphnse_plan* P, sphnse_state* st, const double* forcing, const double* g, NewtonCtl& q) {
    const int n = P->n_coeff;
    Work W = work(P);
    Coef gc;
    for (int j = 0; j < SPHNSE_MAXK; ++j) gc.c[j] = g[j];
    int rc;
    if ((rc = clear_norms(P))) return rc;
    stage_begin(P, SPHNSE_STAGE_STEP);
    k_predict<<<grid(n), 256, 0, P->stream>>>(reinterpret_cast<const double2*>(st->alpha),
                                               reinterpret_cast<const double2*>(st->dif), gc, q.k, W.y0, W.psi, W.d,
                                               W.ynew, fmaxf(float(q.thr), 1e-30f), P->d_norms, n);
    stage_end(P, SPHNSE_STAGE_STEP);
    if ((rc = stage_launch_check(P))) return rc;
    if (newton_graph_ready(P, st, forcing)) {
        *P->h_ctl = q;
        if (cudaMemcpyAsync(P->d_ctl, P->h_ctl, sizeof(NewtonCtl), cudaMemcpyHostToDevice, P->stream) != cudaSuccess ||
            cudaGraphLaunch(P->ng_exec, P->stream) != cudaSuccess ||
            cudaMemcpyAsync(P->h_ctl, P->d_ctl, sizeof(NewtonCtl), cudaMemcpyDeviceToHost, P->stream) != cudaSuccess ||
            cudaStreamSynchronize(P->stream) != cudaSuccess)
            return SPHNSE_E_CUDA;
        q = *P->h_ctl;
        return SPHNSE_OK;
    }
    const int k = q.k;
    for (;;) {
        if ((rc = rhs_device(P, reinterpret_cast<const double*>(W.ynew), forcing,
                             reinterpret_cast<double*>(W.F))))
            return rc;
        if (q.it > 0 && (rc = clear_norms(P))) return rc;
        stage_begin(P, SPHNSE_STAGE_STEP);
        k_newton<<<grid(n), 256, 0, P->stream>>>(
            W.F, reinterpret_cast<const double2*>(st->alpha), W.y0, W.psi, W.d, W.ynew,
            k >= 2 ? reinterpret_cast<const double2*>(st->dif) + size_t(k - 1) * n : nullptr,
            reinterpret_cast<const double2*>(st->dif) + size_t(k) * n, P->d_lm, q.c, q.nu, q.omega, q.thr,
            P->d_norms, n);
        stage_end(P, SPHNSE_STAGE_STEP);
        if ((rc = stage_launch_check(P))) return rc;
        double nv[5];
        bool bad;
        if ((rc = read_newton_norms(P, nv, &bad))) return rc;
        if (newton_control(q, nv, bad)) return SPHNSE_OK;
    }
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

// The controller's inputs and memory for nsteps steps from st.
void ctl_load(const sphnse_plan* P, const sphnse_state* st, int nsteps, sphnse_step_info* info, StepCtl& S) {
    S = StepCtl{};
    S.rtol = P->rtol;
    S.thr = P->atol / P->rtol;
    S.h_max = P->h_max;
    S.maxk = P->max_order;
    S.newton_max = P->newton_max;
    S.fp64 = P->precision == SPHNSE_FP64;
    S.nsteps = nsteps;
    S.nu = P->nu;
    S.omega = P->Omega;
    ndf_constants(P->bdf != 0, S.gamma, S.iga, S.ec);
    S.info = info;
    S.t = st->t;
    S.h = st->h;
    S.t_end = st->t_end;
    S.h_dif = st->h_dif;
    S.rate = st->rate;
    S.miter_h = st->miter_h;
    S.order = st->order;
    S.nconhk = st->nconhk;
    S.havrate = st->havrate;
    S.miter_k = st->miter_k;
    S.status = SPHNSE_OK;
}

void ctl_store(const StepCtl& S, sphnse_state* st) {
    st->t = S.t;
    st->h = S.h;
    st->h_dif = S.h_dif;
    st->rate = S.rate;
    st->miter_h = S.miter_h;
    st->order = S.order;
    st->nconhk = S.nconhk;
    st->havrate = S.havrate;
    st->miter_k = S.miter_k;
}

// nsteps steps with the attempts driven from the host (stage timing on, or no
// step graph): the same controller functions as the device loop.
int steps_host(sphnse_plan* P, sphnse_state* st, const double* forcing, int nsteps, sphnse_step_info* info) {
    StepCtl S;
    ctl_load(P, st, nsteps, info, S);
    int rc = SPHNSE_OK;
    while (S.status == SPHNSE_OK && S.done < S.nsteps) {
        att_begin(S);
        if (S.do_rescale) {
            Mat A;
            std::memcpy(A.a, S.A, sizeof(A.a));
            stage_begin(P, SPHNSE_STAGE_STEP);
            k_rescale<<<grid(P->n_coeff), 256, 0, P->stream>>>(reinterpret_cast<double2*>(st->dif), A, S.k,
                                                               P->n_coeff);
            stage_end(P, SPHNSE_STAGE_STEP);
            if ((rc = stage_launch_check(P))) break;
        }
        if ((rc = corrector(P, st, forcing, S.g, S.nc))) break;
        att_end(S);
        if (S.accept && (rc = accept(P, st, S.k))) break;
    }
    ctl_store(S, st);
    return rc ? rc : S.status;
}

// The whole step loop as one graph: k_step_begin, then a WHILE node over
// attempts whose body is k_prepare, the Newton WHILE node (RHS, update,
// stopping rule) and k_step_next, then k_accept_g.  The loop ends on the
// device after nsteps accepted steps or an error.  Built per (state,
// forcing, precision, nu, Omega); any failure to build leaves the host loop
// in charge.
bool step_graph_ready(sphnse_plan* P, sphnse_state* st, const double* forcing) {
    if (P->sg_failed || P->timing) return false;
    const void* key[4] = {st->alpha, st->dif, forcing,
                          reinterpret_cast<const void*>(uintptr_t(P->precision) | (uintptr_t(P->coriolis_split) << 8))};
    if (P->sg_exec && std::equal(key, key + 4, P->sg_key) && P->sg_nu == P->nu && P->sg_omega == P->Omega) return true;
    if (P->sg_exec) {
        cudaGraphExecDestroy(P->sg_exec);
        P->sg_exec = nullptr;
    }
    if ((!P->d_step && (cudaMalloc(reinterpret_cast<void**>(&P->d_step), sizeof(StepCtl)) != cudaSuccess ||
                        cudaMallocHost(reinterpret_cast<void**>(&P->h_step), sizeof(StepCtl)) != cudaSuccess)) ||
        (!P->cap_stream && cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking) != cudaSuccess)) {
        cudaGetLastError();
        P->sg_failed = true;
        return false;
    }
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return false;
    Work W = work(P);
    const int n = P->n_coeff;
    double2* alpha = reinterpret_cast<double2*>(st->alpha);
    double2* dif = reinterpret_cast<double2*>(st->dif);
    const cudaStream_t cs = P->cap_stream;
    // add a conditional WHILE node to the graph under capture on cs, make it
    // the capture's only dependency and return its body graph (null on failure)
    auto add_while = [cs](cudaGraphConditionalHandle h) -> cudaGraph_t {
        cudaStreamCaptureStatus status;
        cudaGraph_t capg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        if (cudaStreamGetCaptureInfo(cs, &status, nullptr, &capg, &deps, nullptr, &ndeps) != cudaSuccess ||
            status != cudaStreamCaptureStatusActive)
            return nullptr;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, capg, deps, nullptr, ndeps, &cp) != cudaSuccess ||
            cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
            return nullptr;
        return cp.conditional.phGraph_out[0];
    };
    auto begin = [cs](cudaGraph_t gr) {
        return gr && cudaStreamBeginCaptureToGraph(cs, gr, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) ==
                         cudaSuccess;
    };
    auto end = [cs]() {
        cudaGraph_t out = nullptr;
        return cudaStreamEndCapture(cs, &out) == cudaSuccess;
    };
    const cudaStream_t saved = P->stream;
    P->stream = cs;
    cudaGraph_t g = nullptr, body = nullptr, inner = nullptr;
    cudaGraphConditionalHandle hloop, hnewton;
    // the top level: begin, the attempt loop, the last accept
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&hloop, g, 1, cudaGraphCondAssignDefault) == cudaSuccess && begin(g);
    if (ok) {
        k_step_begin<<<1, 32, 0, cs>>>(P->d_step, P->d_norms);
        body = add_while(hloop);
        k_accept_g<<<grid(n), 256, 0, cs>>>(dif, W.d, alpha, W.ynew, P->d_step, n);
        ok = end() && body;
    }
    // one attempt: prepare, the Newton loop, the controller
    ok = ok && cudaGraphConditionalHandleCreate(&hnewton, body, 1, cudaGraphCondAssignDefault) == cudaSuccess &&
         begin(body);
    if (ok) {
        k_prepare<<<grid(n), 256, 0, cs>>>(alpha, dif, W.y0, W.psi, W.d, W.ynew, P->d_step, P->d_norms, hnewton, n);
        inner = add_while(hnewton);
        k_step_next<<<1, 32, 0, cs>>>(P->d_step, P->d_norms, hloop);
        ok = end() && inner;
    }
    // one Newton iteration: RHS at ynew, update, stopping rule
    ok = ok && begin(inner);
    if (ok) {
        const int rc = rhs_device(P, reinterpret_cast<const double*>(W.ynew), forcing, reinterpret_cast<double*>(W.F));
        k_newton_g<<<grid(n), 256, 0, cs>>>(W.F, alpha, W.y0, W.psi, W.d, W.ynew, dif, P->d_lm, &P->d_step->nc,
                                            P->d_norms, n, hnewton);
        ok = end() && rc == SPHNSE_OK;
    }
    P->stream = saved;
    if (ok) ok = cudaGraphInstantiate(&P->sg_exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();   // a failed capture leaves no sticky error; clear the last one
    if (!ok) {
        P->sg_exec = nullptr;
        P->sg_failed = true;
        return false;
    }
    std::copy(key, key + 4, P->sg_key);
    P->sg_nu = P->nu;
    P->sg_omega = P->Omega;
    return true;
}

// nsteps steps in one launch of the step graph: the controller's state goes
// up before and comes back after it (one host synchronisation per call).
int steps_graph(sphnse_plan* P, sphnse_state* st, int nsteps, sphnse_step_info* info) {
    if (info && nsteps > P->info_cap) {
        if (P->d_info) cudaFree(P->d_info);
        if (P->h_info) cudaFreeHost(P->h_info);
        P->d_info = P->h_info = nullptr;
        P->info_cap = 0;
        const size_t bytes = size_t(nsteps) * sizeof(sphnse_step_info);
        if (cudaMalloc(reinterpret_cast<void**>(&P->d_info), bytes) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void**>(&P->h_info), bytes) != cudaSuccess) {
            cudaGetLastError();
            return SPHNSE_E_NOMEM;
        }
        P->info_cap = nsteps;
    }
    StepCtl& S = *P->h_step;
    ctl_load(P, st, nsteps, info ? P->d_info : nullptr, S);
    if (cudaMemcpyAsync(P->d_step, P->h_step, sizeof(StepCtl), cudaMemcpyHostToDevice, P->stream) != cudaSuccess ||
        cudaGraphLaunch(P->sg_exec, P->stream) != cudaSuccess ||
        cudaMemcpyAsync(P->h_step, P->d_step, sizeof(StepCtl), cudaMemcpyDeviceToHost, P->stream) != cudaSuccess ||
        (info && cudaMemcpyAsync(P->h_info, P->d_info, size_t(nsteps) * sizeof(sphnse_step_info),
                                 cudaMemcpyDeviceToHost, P->stream) != cudaSuccess) ||
        cudaStreamSynchronize(P->stream) != cudaSuccess)
        return SPHNSE_E_CUDA;
    ctl_store(S, st);
    if (info) std::memcpy(info, P->h_info, size_t(S.done) * sizeof(sphnse_step_info));   // entries of accepted steps
    return S.status;
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
    return sphnse_advance(P, st, forcing, 1, info);
}

int sphnse_advance(sphnse_plan* P, sphnse_state* st, const double* forcing, int nsteps, sphnse_step_info* info) {
    if (!P || !st || !st->alpha || !st->dif || nsteps < 0) return SPHNSE_E_ARG;
    if (nsteps == 0) return SPHNSE_OK;
    if (step_graph_ready(P, st, forcing)) return steps_graph(P, st, nsteps, info);
    return steps_host(P, st, forcing, nsteps, info);
}

int sphnse_replay_step(sphnse_plan* P, sphnse_state* st, const double* forcing, double h, int k, int newton_max,
                       sphnse_step_info* info) {
    if (!P || !st || !(h > 0.0) || k < 1 || k > SPHNSE_MAXK || newton_max < 1) return SPHNSE_E_ARG;
    const NDFConst C(P->bdf != 0);
    const double h_dif_before = st->h_dif;
    st->order = k;
    int rc;
    if ((rc = rescale(P, st, h, k))) return rc;
    if (h != st->miter_h || k != st->miter_k) {
        st->havrate = 0;
        st->miter_h = h;
        st->miter_k = k;
    }
    double g[SPHNSE_MAXK];
    for (int j = 0; j < SPHNSE_MAXK; ++j) g[j] = j < k ? C.gamma[j] * C.iga[k - 1] : 0.0;
    NewtonCtl q;
    newton_init(q, h * C.iga[k - 1], P->nu, P->Omega, P->atol / P->rtol, P->rtol, st->rate, st->havrate, k,
                newton_max, 1, P->precision == SPHNSE_FP64);
    if ((rc = corrector(P, st, forcing, g, q))) return rc;
    if (q.nonfinite) return SPHNSE_E_NONFINITE;
    st->rate = q.rate;
    st->havrate = q.havrate;
    if ((rc = accept(P, st, k))) return rc;
    st->t += h;
    st->h = h;
    if (info) {
        info->t = st->t;
        info->h = h;
        info->err = q.nrm[1] * C.ec[k - 1];
        info->order = k;
        info->newton_iters = q.its;
        info->rejections = 0;
        info->rhs_evals = q.its;
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

int sphnse_adjoint_step_explicit(sphnse_plan* P, double h, int k, double h_dif_before, const double* alpha_next,
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
