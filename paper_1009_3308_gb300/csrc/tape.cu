// Checkpointed trajectory tape and the tape-driven reverse NDF step.
//
// The differentiated map is the replay of a fixed step schedule [(h_n, k_n)]
// (frozen controller, corrector iterated to convergence; Sec. 4.2,
// Eq. (ode_disc)).  Recording runs the replay steps on a tape-owned state and
// keeps every C-th state (alpha, differences, controller scalars) in
// tape-owned device memory.  The reverse sweep asks for steps n-1, n-2, ..., 0;
// the first request inside a segment of C steps replays that segment from its
// checkpoint and keeps the states it produces, so a trajectory of n steps
// costs n + n forward steps and holds ceil(n / C) checkpoints + C states.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "internal.h"

struct sphnse_tape {
    sphnse_plan* plan = nullptr;
    int n = 0;            // n_coeff
    int max_steps = 0;
    int every = 0;        // checkpoint interval C
    int nck = 0;          // checkpoint slots
    // recorded trajectory
    bool begun = false;
    int nsteps = 0;
    double t0 = 0, h0 = 0, nu = 0, omega = 0;
    int precision = 0, bdf = 0;
    const double* forcing = nullptr;   // caller-owned, steady over the trajectory
    std::vector<double> h, hdif;
    std::vector<int> k, newton_max;
    std::vector<sphnse_state> ck_st;   // controller scalars at each checkpoint
    sphnse_state st{};                 // the forward state (points into cur_*)
    // reverse sweep
    int next_rev = -1;    // the step index the next reverse call must name
    int seg_cached = -1;  // segment whose states seg[] holds
    // device memory: one allocation carved into the arrays below
    void* base = nullptr;
    double2* alpha0 = nullptr;     // n
    double2* cur = nullptr;        // alpha n, then dif (MAXK + 2) n
    double2* ck = nullptr;         // nck x (MAXK + 3) n
    double2* rs = nullptr;         // recompute state (MAXK + 3) n
    double2* seg = nullptr;        // C x n: alpha after each step of the cached segment
    double2* dbar = nullptr;       // (MAXK + 2) n: adjoint of the differences
};

namespace {

constexpr int kRows = SPHNSE_MAXK + 3;   // alpha + (MAXK + 2) difference rows

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? SPHNSE_OK : SPHNSE_E_CUDA; }

int copy_dev(sphnse_tape* T, void* dst, const void* src, size_t rows) {
    return cuda_rc(cudaMemcpyAsync(dst, src, rows * size_t(T->n) * sizeof(double2), cudaMemcpyDeviceToDevice,
                                   T->plan->stream));
}

// The plan must still describe the map the tape recorded.
bool same_map(const sphnse_tape* T) {
    const sphnse_plan* P = T->plan;
    return P->nu == T->nu && P->Omega == T->omega && P->precision == T->precision && P->bdf == T->bdf;
}

// Replay segment s from its checkpoint into seg[] (states after each step).
int load_segment(sphnse_tape* T, int s) {
    if (T->seg_cached == s) return SPHNSE_OK;
    const size_t rows = kRows;
    int rc;
    if ((rc = copy_dev(T, T->rs, T->ck + size_t(s) * rows * T->n, rows))) return rc;
    sphnse_state st = T->ck_st[s];
    st.alpha = reinterpret_cast<double*>(T->rs);
    st.dif = reinterpret_cast<double*>(T->rs + T->n);
    const int lo = s * T->every, hi = std::min(T->nsteps, lo + T->every);
    for (int i = lo; i < hi; ++i) {
        if ((rc = sphnse_replay_step(T->plan, &st, T->forcing, T->h[i], T->k[i], T->newton_max[i], nullptr)))
            return rc;
        if ((rc = copy_dev(T, T->seg + size_t(i - lo) * T->n, T->rs, 1))) return rc;
    }
    T->seg_cached = s;
    return SPHNSE_OK;
}

}  // namespace

extern "C" {

int sphnse_tape_create(sphnse_plan* P, int max_steps, int checkpoint_every, sphnse_tape** out) {
    if (!out) return SPHNSE_E_ARG;
    *out = nullptr;
    if (!P || max_steps < 1 || checkpoint_every < 1) return SPHNSE_E_ARG;
    sphnse_tape* T = new (std::nothrow) sphnse_tape();
    if (!T) return SPHNSE_E_NOMEM;
    T->plan = P;
    T->n = P->n_coeff;
    T->max_steps = max_steps;
    T->every = std::min(checkpoint_every, max_steps);
    T->nck = (max_steps + T->every - 1) / T->every;
    const size_t n = T->n;
    const size_t total = n * (1 + kRows + size_t(T->nck) * kRows + kRows + size_t(T->every) + (kRows - 1));
    int dev_prev = 0;
    cudaGetDevice(&dev_prev);
    cudaSetDevice(P->device);
    const cudaError_t e = cudaMalloc(&T->base, total * sizeof(double2));
    cudaSetDevice(dev_prev);
    if (e != cudaSuccess) {
        delete T;
        return SPHNSE_E_NOMEM;
    }
    double2* p = static_cast<double2*>(T->base);
    T->alpha0 = p;
    p += n;
    T->cur = p;
    p += kRows * n;
    T->ck = p;
    p += size_t(T->nck) * kRows * n;
    T->rs = p;
    p += kRows * n;
    T->seg = p;
    p += size_t(T->every) * n;
    T->dbar = p;
    T->h.reserve(max_steps);
    T->hdif.reserve(max_steps);
    T->k.reserve(max_steps);
    T->newton_max.reserve(max_steps);
    T->ck_st.resize(T->nck);
    *out = T;
    return SPHNSE_OK;
}

void sphnse_tape_destroy(sphnse_tape* T) {
    if (!T) return;
    if (T->base) {
        cudaStreamSynchronize(T->plan->stream);
        cudaFree(T->base);
    }
    delete T;
}

int sphnse_tape_begin(sphnse_tape* T, const double* alpha0, double t0, double h0, const double* forcing) {
    if (!T || !alpha0 || !std::isfinite(t0)) return SPHNSE_E_ARG;
    sphnse_plan* P = T->plan;
    int rc;
    if ((rc = copy_dev(T, T->alpha0, alpha0, 1))) return rc;
    if ((rc = copy_dev(T, T->cur, alpha0, 1))) return rc;
    T->st = sphnse_state{};
    T->st.alpha = reinterpret_cast<double*>(T->cur);
    T->st.dif = reinterpret_cast<double*>(T->cur + T->n);
    T->st.t_end = INFINITY;
    if ((rc = sphnse_state_init(P, &T->st, t0, h0, forcing))) return rc;
    T->t0 = t0;
    T->h0 = T->st.h;
    T->nu = P->nu;
    T->omega = P->Omega;
    T->precision = P->precision;
    T->bdf = P->bdf;
    T->forcing = forcing;
    T->nsteps = 0;
    T->h.clear();
    T->hdif.clear();
    T->k.clear();
    T->newton_max.clear();
    T->next_rev = -1;
    T->seg_cached = -1;
    T->begun = true;
    return SPHNSE_OK;
}

int sphnse_tape_record(sphnse_tape* T, double h, int k, int newton_max, sphnse_step_info* info) {
    if (!T || !T->begun || !(h > 0.0) || k < 1 || k > SPHNSE_MAXK || newton_max < 1) return SPHNSE_E_ARG;
    if (T->nsteps >= T->max_steps) return SPHNSE_E_TOO_LARGE;
    if (!same_map(T)) return SPHNSE_E_ARG;
    int rc;
    const int i = T->nsteps;
    if (i % T->every == 0) {
        const int s = i / T->every;
        if ((rc = copy_dev(T, T->ck + size_t(s) * kRows * T->n, T->cur, kRows))) return rc;
        T->ck_st[s] = T->st;
    }
    sphnse_step_info loc{};
    if ((rc = sphnse_replay_step(T->plan, &T->st, T->forcing, h, k, newton_max, &loc))) return rc;
    T->h.push_back(h);
    T->k.push_back(k);
    T->newton_max.push_back(newton_max);
    T->hdif.push_back(loc.h_dif_before);
    T->nsteps = i + 1;
    T->next_rev = -1;
    T->seg_cached = -1;
    if (info) *info = loc;
    return SPHNSE_OK;
}

int sphnse_tape_info(const sphnse_tape* T, int* nsteps, double* t, double* h0) {
    if (!T) return SPHNSE_E_ARG;
    if (nsteps) *nsteps = T->nsteps;
    if (t) *t = T->st.t;
    if (h0) *h0 = T->h0;
    return SPHNSE_OK;
}

int sphnse_tape_state(const sphnse_tape* T, double* alpha_out) {
    if (!T || !T->begun || !alpha_out) return SPHNSE_E_ARG;
    return cuda_rc(cudaMemcpyAsync(alpha_out, T->cur, size_t(T->n) * sizeof(double2), cudaMemcpyDeviceToDevice,
                                   T->plan->stream));
}

int sphnse_adjoint_step(sphnse_plan* P, sphnse_tape* T, int step_index, double* lambda, double* dJ_dnu) {
    if (!P || !T || T->plan != P || !lambda || !T->begun) return SPHNSE_E_ARG;
    if (step_index < 0 || step_index >= T->nsteps) return SPHNSE_E_ARG;
    if (!same_map(T)) return SPHNSE_E_ARG;
    int rc;
    if (step_index == T->nsteps - 1) {
        // a new reverse sweep: the final differences do not enter the objective
        if ((rc = cuda_rc(cudaMemsetAsync(T->dbar, 0, size_t(SPHNSE_MAXK + 2) * T->n * sizeof(double2),
                                          P->stream))))
            return rc;
    } else if (step_index != T->next_rev) {
        return SPHNSE_E_ARG;
    }
    const int s = step_index / T->every;
    if ((rc = load_segment(T, s))) return rc;
    const double* alpha_next = reinterpret_cast<const double*>(T->seg + size_t(step_index - s * T->every) * T->n);
    double nub = 0.0;
    double* dbar = reinterpret_cast<double*>(T->dbar);
    if ((rc = sphnse_adjoint_step_explicit(P, T->h[step_index], T->k[step_index], T->hdif[step_index], alpha_next,
                                           lambda, dbar, &nub)))
        return rc;
    if (step_index == 0 &&
        (rc = sphnse_adjoint_init(P, T->h0, reinterpret_cast<const double*>(T->alpha0), lambda, dbar, &nub)))
        return rc;
    if (dJ_dnu) *dJ_dnu += nub;
    T->next_rev = step_index - 1;
    return SPHNSE_OK;
}

int sphnse_adjoint_run(sphnse_plan* P, sphnse_tape* T, double* lambda, double* dJ_dnu) {
    if (!P || !T || !T->begun || T->nsteps < 1) return SPHNSE_E_ARG;
    for (int i = T->nsteps - 1; i >= 0; --i) {
        const int rc = sphnse_adjoint_step(P, T, i, lambda, dJ_dnu);
        if (rc) return rc;
    }
    return SPHNSE_OK;
}

}  // extern "C"
