// The NDF step controller (Sec. 4.2): constants of the scheme, the
// difference rescaling matrix, the simplified-Newton stopping rule and the
// attempt start / finish with step rejection and order / step selection.
// Host-and-device functions on a StepCtl: the single-plan step loop (one
// thread of a graph-launched kernel, or the host) and the ensemble's
// per-instance rounds take their decisions with the same code.
#pragma once
#include <cmath>

#include "internal.h"

namespace sph {

// NDF coefficients kappa_k (Sec. 4.2; kappa = 0: BDF), gamma_k = sum_{j<=k}
// 1/j, iga_k = 1 / ((1 - kappa_k) gamma_k) and the error constants
// ec_k = kappa_k gamma_k + 1 / (k + 1)
inline void ndf_constants(bool bdf, double* gamma, double* iga, double* ec) {
    const double kappa[SPHNSE_MAXK] = {-0.1850, -1.0 / 9.0, -0.0823, -0.0415, 0.0};
    double g = 0.0;
    for (int k = 1; k <= SPHNSE_MAXK; ++k) {
        const double kp = bdf ? 0.0 : kappa[k - 1];
        g += 1.0 / k;
        gamma[k - 1] = g;
        iga[k - 1] = 1.0 / (g * (1.0 - kp));
        ec[k - 1] = kp * g + 1.0 / (k + 1.0);
    }
}

// (R(rho) U)[:k, :k], R_ij = prod_{l=1..i} (l - 1 - j rho) / l, U = R(1),
// into A (row-major SPHNSE_MAXK x SPHNSE_MAXK, zero outside k x k)
__host__ __device__ inline void rescale_matrix_into(int k, double rho, double* A) {
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
    for (int i = 0; i < SPHNSE_MAXK * SPHNSE_MAXK; ++i) A[i] = 0.0;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += R[i][l] * U[l][j];
            A[i * SPHNSE_MAXK + j] = s;
        }
}

// Corrector parameters of one attempt (tight: iterate to the rounding level,
// for the replay).
__host__ __device__ inline void newton_init(NewtonCtl& q, double c, double nu, double omega, double thr, double rtol,
                                            double rate, int havrate, int k, int maxit, int tight, int fp64) {
    q = NewtonCtl{};
    q.c = c;
    q.nu = nu;
    q.omega = omega;
    q.thr = thr;
    q.rtol = rtol;
    q.rate = rate;
    q.havrate = havrate;
    q.k = k;
    q.maxit = maxit;
    q.tight = tight;
    q.fp64 = fp64;
}

// The corrector's stopping rule after iteration q.it, from the norms of that
// iteration (nv[0..3]: the slots of the Newton update, nv[4]: the predictor's
// scale, read at the first iteration).  Convergence and rate tests of the
// MATLAB ODE suite's simplified Newton; returns true when the loop stops.
__host__ __device__ inline bool newton_control(NewtonCtl& q, const double* nv, bool nonfinite) {
    const double eps = 2.220446049250313e-16;
    const int it = q.it;
    bool stop = false, conv = false;
    if (nonfinite) {
        q.nonfinite = 1;
        stop = true;
    } else {
        if (it == 0) q.ynorm = nv[4];
        q.its = it + 1;
        for (int j = 0; j < 4; ++j) q.nrm[j] = nv[j];
        const double newnrm = nv[0], minnrm = 100.0 * eps * q.ynorm, oldnrm = q.oldnrm;
        const double rtol = q.rtol;
        if (q.tight) {
            // converged to the rounding level: below 1e-15 in the weighted
            // norm, or no longer shrinking (FP32 / BF16 contractions stall at
            // their own rounding level long before 1e-15)
            const bool stalled = !q.fp64 && it >= 3 && newnrm > 0.8 * oldnrm;
            if (newnrm <= fmax(minnrm, 1e-15) || stalled) stop = conv = true;
        } else if (newnrm <= minnrm) {
            stop = conv = true;
        } else if (it == 0) {
            if (q.havrate) {
                const double errit = newnrm * q.rate / (1.0 - q.rate);
                if (errit <= 0.05 * rtol) stop = conv = true;
            } else {
                q.rate = 0.0;
            }
        } else if (newnrm > 0.9 * oldnrm) {
            stop = true;   // too slow
        } else {
            q.rate = fmax(0.9 * q.rate, newnrm / oldnrm);
            q.havrate = 1;
            const double errit = newnrm * q.rate / (1.0 - q.rate);
            if (errit <= 0.5 * rtol) stop = conv = true;
            else if (it == q.maxit - 1) stop = true;
            else if (0.5 * rtol < errit * pow(q.rate, double(q.maxit - 1 - it))) stop = true;
        }
        q.oldnrm = newnrm;
        if (!stop && it + 1 >= q.maxit) {
            stop = true;
            conv = q.tight != 0;   // a tight loop that ran out counts as converged
        }
    }
    q.it = it + 1;
    q.conv = conv;
    q.stop = stop;
    return stop;
}

constexpr double EPS16 = 16.0 * 2.220446049250313e-16;

// Start an attempt: clamp h to [16 eps |t|, h_max] and to t_end, rescale the
// differences to it if it changed, reset the rate memory on a new (h, k) and
// set the predictor weights and the corrector's parameters.
__host__ __device__ inline void att_begin(StepCtl& S) {
    if (S.attempt == 0) {
        S.h_dif_before = S.h_dif;
        S.nofailed = 1;
        S.rejections = 0;
        S.newton_total = 0;
        S.rhs_evals = 0;
    }
    const double hmin = EPS16 * fabs(S.t);
    double h = fmin(S.h_max, fmax(hmin, S.h));
    if (1.1 * h >= S.t_end - S.t) h = S.t_end - S.t;
    S.h = h;
    S.h_att = h;
    const int k = S.order;
    S.k = k;
    S.do_rescale = h != S.h_dif;
    if (S.do_rescale) {
        rescale_matrix_into(k, h / S.h_dif, S.A);
        S.h_dif = h;
        S.nconhk = 0;
    }
    if (h != S.miter_h || k != S.miter_k) {
        S.havrate = 0;
        S.miter_h = h;
        S.miter_k = k;
    }
    for (int j = 0; j < SPHNSE_MAXK; ++j) S.g[j] = j < k ? S.gamma[j] * S.iga[k - 1] : 0.0;
    newton_init(S.nc, h * S.iga[k - 1], S.nu, S.omega, S.thr, S.rtol, S.rate, S.havrate, k, S.newton_max, 0, S.fp64);
}

// The accepted step's record (t, h, order, error estimate, the step's Newton
// iterations and rejections, the next order and step size).
__host__ __device__ inline void fill_info(const StepCtl& S, sphnse_step_info& I) {
    I.t = S.t;
    I.h = S.h_att;
    I.err = S.err;
    I.order = S.k_acc;
    I.newton_iters = S.newton_total;
    I.rejections = S.rejections;
    I.rhs_evals = S.rhs_evals;
    I.next_order = S.order;
    I.next_h = S.h;
    I.h_dif_before = S.h_dif_before;
}

// Finish an attempt from the corrector's results: reject (a smaller h, maybe
// a lower order) or accept (advance t, record the step, choose the next
// order and step size from the error estimates of orders k - 1, k, k + 1).
__host__ __device__ inline void att_end(StepCtl& S) {
    const NewtonCtl& q = S.nc;
    S.rate = q.rate;
    S.havrate = q.havrate;
    S.accept = 0;
    if (q.nonfinite) {
        S.status = SPHNSE_E_NONFINITE;
        return;
    }
    const int k = S.k;
    const double h = S.h_att, hmin = EPS16 * fabs(S.t);
    S.newton_total += q.its;
    S.rhs_evals += q.its;
    const double err = q.nrm[1] * S.ec[k - 1];
    if (!q.conv || err > S.rtol) {
        ++S.rejections;
        if (h <= hmin) {
            S.status = SPHNSE_E_STEP_TOO_SMALL;
            return;
        }
        if (!q.conv) {
            S.h = fmax(hmin, 0.3 * h);
        } else if (S.nofailed) {
            S.nofailed = 0;
            double hopt = h * fmax(0.1, 0.833 * pow(S.rtol / err, 1.0 / (k + 1)));
            if (k > 1) {
                const double errkm1 = q.nrm[2] * S.ec[k - 2];
                const double hkm1 = h * fmax(0.1, 0.769 * pow(S.rtol / errkm1, 1.0 / k));
                if (hkm1 > hopt) {
                    hopt = fmin(h, hkm1);
                    S.order = k - 1;
                }
            }
            S.h = fmax(hmin, hopt);
        } else {
            S.h = fmax(hmin, 0.5 * h);
        }
        if (++S.attempt >= 200) S.status = SPHNSE_E_STEP_TOO_SMALL;
        return;
    }
    // accepted
    S.accept = 1;
    S.k_acc = k;
    S.t += h;
    S.nconhk = S.nconhk + 1 < SPHNSE_MAXK + 2 ? S.nconhk + 1 : SPHNSE_MAXK + 2;
    if (S.nconhk >= k + 2) {
        double temp = 1.2 * pow(err / S.rtol, 1.0 / (k + 1));
        double hopt = temp > 0.1 ? h / temp : 10.0 * h;
        int kopt = k;
        if (k > 1) {
            const double errkm1 = q.nrm[2] * S.ec[k - 2];
            temp = 1.3 * pow(errkm1 / S.rtol, 1.0 / k);
            const double hkm1 = temp > 0.1 ? h / temp : 10.0 * h;
            if (hkm1 > hopt) {
                hopt = hkm1;
                kopt = k - 1;
            }
        }
        if (k < S.maxk) {
            const double errkp1 = q.nrm[3] * S.ec[k];
            temp = 1.4 * pow(errkp1 / S.rtol, 1.0 / (k + 2));
            const double hkp1 = temp > 0.1 ? h / temp : 10.0 * h;
            if (hkp1 > hopt) {
                hopt = hkp1;
                kopt = k + 1;
            }
        }
        if (hopt > h) {
            S.h = hopt;
            if (kopt != k) {
                S.order = kopt;
                S.nconhk = 0;
            }
        }
    }
    S.err = err;
    S.sum_newton += S.newton_total;
    S.sum_rejections += S.rejections;
    if (S.info) fill_info(S, S.info[S.done]);
    ++S.done;
    S.attempt = 0;
}

}  // namespace sph
