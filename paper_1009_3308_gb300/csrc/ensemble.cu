// Batched ensemble of independent problems (uneven truncation degrees and
// viscosities) advanced together.
//
// Instances are bucketed by truncation L; each bucket shares one plan (its
// Legendre tables) and runs every RHS stage as ONE launch over all of its
// instances (items (instance, m) for the streaming Legendre kernels, a grid
// dimension for the others), so that the table rows of an order are streamed
// once per bucket and reused across instances through L2.  The batched RHS of
// all buckets plus the batched Newton update are captured once into a CUDA
// graph and replayed as a single launch per Newton iteration.
//
// Time stepping: every instance keeps its own adaptive NDF controller (step
// size, order, Newton rate; the same quasi-constant step-size scheme as
// sphnse_step, Sec. 4.2 Eq. (ode_disc)).  The instances advance
// asynchronously in rounds: one round is one captured graph -- accept of the
// previous step, rescale and predictor of a new attempt, one batched RHS and
// one Newton update -- in which every instance does whatever its own
// controller is at (flag bits in a per-instance parameter array), followed by
// one read of all instances' norms.  An instance that converges, rejects or
// accepts starts its next attempt in the next round, so no instance waits for
// another's rejected attempts or extra Newton iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "internal.h"
#include "dmath.cuh"
#include "newton.cuh"
#include "reduce.cuh"

namespace sph {
namespace {

constexpr double EPS = 2.220446049250313e-16;
const double KAPPA_E[SPHNSE_MAXK] = {-0.1850, -1.0 / 9.0, -0.0823, -0.0415, 0.0};

// flag bits of InstPar::flags: what an instance does in the current launch
constexpr int F_INIT = 1;       // initial weight norm of F and zeroed differences
constexpr int F_ACCEPT = 2;     // apply the step accepted in the previous round (order ka)
constexpr int F_RESCALE = 4;    // rescale the differences to a new step size
constexpr int F_PREDICT = 8;    // predictor of a new attempt (and the weight norm of alpha)
constexpr int F_NEWTON = 16;    // one simplified-Newton update at the batched RHS

struct InstPar {
    long off;      // offset (complex entries) of this instance in the concatenated vectors
    int n;         // packed entries
    int k;         // order of the current attempt
    int flags;     // F_* bits for the current launch
    int ka;        // order of the step accepted by F_ACCEPT
    double c;      // h * iga_k
    double nu, Omega, thr;
    const int2* lm;
    double g[SPHNSE_MAXK];
    double A[SPHNSE_MAXK * SPHNSE_MAXK];
    double h0;     // initial step (init kernel)
};

// One 256-thread block per (instance, 256 consecutive entries): the block
// table btab lists (instance, block of the instance), so no block is empty
// and a block never spans two instances (the norm reductions are per block).
constexpr int EB = 256;

#define INST_PROLOGUE_ALL(FLAG)                              \
    const int2 bt = btab[blockIdx.x];                        \
    const InstPar& p = par[bt.x];                            \
    if (!(p.flags & (FLAG))) return;                         \
    const int i = bt.y * EB + threadIdx.x;                   \
    const long o = p.off;

#define INST_PROLOGUE(FLAG)                                  \
    INST_PROLOGUE_ALL(FLAG)                                  \
    if (i >= p.n) return;

__global__ void kb_wnorm(const int2* btab, const InstPar* par, int flag, const double2* v, const double2* y,
                         unsigned long long* norms, int slot) {
    INST_PROLOGUE_ALL(flag)
    double r[1] = {0.0};
    if (i < p.n) {
        const double2 a = v[o + i], b = y[o + i];
        r[0] = fmax(fabs(a.x) * rcp64<1>(fmax(fabs(b.x), p.thr)), fabs(a.y) * rcp64<1>(fmax(fabs(b.y), p.thr)));
    }
    const int id[1] = {slot};
    block_amax<1>(norms + 8 * bt.x, r, id);
}

__global__ void kb_init(const int2* btab, const InstPar* par, double2* dif, const double2* F) {
    INST_PROLOGUE(F_INIT)
    const double2 f = F[o + i];
    double2* D = dif + 7 * o;
    D[i] = make_double2(p.h0 * f.x, p.h0 * f.y);
    for (int j = 1; j < SPHNSE_MAXK + 2; ++j) D[size_t(j) * p.n + i] = make_double2(0.0, 0.0);
}

__global__ void kb_rescale(const int2* btab, const InstPar* par, double2* dif) {
    INST_PROLOGUE(F_RESCALE)
    double2* D = dif + 7 * o;
    double2 old[SPHNSE_MAXK];
    for (int j = 0; j < p.k; ++j) old[j] = D[size_t(j) * p.n + i];
    for (int j = 0; j < p.k; ++j) {
        double sx = 0.0, sy = 0.0;
        for (int l = 0; l < p.k; ++l) {
            const double a = p.A[l * SPHNSE_MAXK + j];
            sx += a * old[l].x;
            sy += a * old[l].y;
        }
        D[size_t(j) * p.n + i] = make_double2(sx, sy);
    }
}

__global__ void kb_predict(const int2* btab, const InstPar* par, const double2* y, const double2* dif, double2* y0,
                           double2* psi, double2* d, double2* ynew, unsigned long long* norms) {
    INST_PROLOGUE_ALL(F_PREDICT)
    float r[1] = {0.f};
    if (i < p.n) {
        const double2* D = dif + 7 * o;
        const double2 yi = y[o + i];
        double2 a = yi, q = make_double2(0.0, 0.0);
        for (int j = 0; j < p.k; ++j) {
            const double2 dj = D[size_t(j) * p.n + i];
            a.x += dj.x;
            a.y += dj.y;
            q.x += p.g[j] * dj.x;
            q.y += p.g[j] * dj.y;
        }
        y0[o + i] = a;
        ynew[o + i] = a;
        psi[o + i] = q;
        d[o + i] = make_double2(0.0, 0.0);
        // slot 4: ||y / max(|y|, thr)||_inf (FP32, as the corrector's norms)
        const float thr = fmaxf(float(p.thr), 1e-30f), ax = absf_trunc(yi.x), ay = absf_trunc(yi.y);
        r[0] = fmaxf(ax / fmaxf(ax, thr), ay / fmaxf(ay, thr));
    }
    const int id[1] = {4};
    block_amax_f<1>(norms + 8 * bt.x, r, id, false);
}

__global__ void kb_newton(const int2* btab, const InstPar* par, const double2* F, const double2* y,
                          const double2* y0, const double2* psi, double2* d, double2* ynew, const double2* dif,
                          unsigned long long* norms) {
    INST_PROLOGUE_ALL(F_NEWTON)
    float nv[4] = {0.f, 0.f, 0.f, 0.f};
    bool bad = false;
    if (i < p.n) {
        const int2 q = p.lm[i];
        const double2* D = dif + 7 * o;
        const NewtonEntry e = newton_entry(q.x, q.y, p.c, float(p.nu), float(2.0 * p.Omega), fmaxf(float(p.thr), 1e-30f),
                                           F[o + i], psi[o + i], d[o + i], y[o + i], ynew[o + i], y0[o + i],
                                           p.k >= 2 ? D + size_t(p.k - 1) * p.n + i : nullptr,
                                           D[size_t(p.k) * p.n + i]);
        d[o + i] = e.dn;
        ynew[o + i] = e.yv;
        for (int j = 0; j < 4; ++j) nv[j] = e.nv[j];
        bad = e.bad;
    }
    const int id[4] = {0, 1, 2, 3};
    block_amax_f<4>(norms + 8 * bt.x, nv, id, bad);
}

__global__ void kb_accept(const int2* btab, const InstPar* par, double2* dif, const double2* d, double2* y,
                          const double2* ynew) {
    INST_PROLOGUE(F_ACCEPT)
    double2* D = dif + 7 * o;
    const int k = p.ka;
    const double2 dd = d[o + i], dk = D[size_t(k) * p.n + i];
    D[size_t(k + 1) * p.n + i] = make_double2(dd.x - dk.x, dd.y - dk.y);
    double2 up = dd;
    D[size_t(k) * p.n + i] = dd;
    for (int j = k - 1; j >= 0; --j) {
        double2 v = D[size_t(j) * p.n + i];
        v.x += up.x;
        v.y += up.y;
        D[size_t(j) * p.n + i] = v;
        up = v;
    }
    y[o + i] = ynew[o + i];
}

// (R(rho) U)[:k, :k]
void rescale_mat(int k, double rho, double* A) {
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
    std::memset(A, 0, sizeof(double) * SPHNSE_MAXK * SPHNSE_MAXK);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += R[i][l] * U[l][j];
            A[i * SPHNSE_MAXK + j] = s;
        }
}

struct Ctl {
    double t = 0, h = 0, h_dif = 0, rate = 0, miter_h = 0;
    int k = 1, nconhk = 0, havrate = 0, miter_k = 0;
    // per step
    bool done = false, nofailed = true;
    int rejections = 0, newton = 0;
    double h_dif_before = 0, hmin = 0, ha = 0;
    int ka = 1;
    // per attempt
    bool attempting = false, in_newton = false, conv = false;
    int its = 0;
    double oldnrm = 0, ynorm = 0, nrm[4] = {0, 0, 0, 0};
    // asynchronous rounds
    int state = 0;                // S_IDLE, S_START (new attempt next round), S_NEWTON
    int it = 0;                   // Newton iteration of the current attempt
    int steps_left = 0, attempts = 0;
    bool pending_accept = false;  // F_ACCEPT in the next launch
    int acc_k = 1;
};

constexpr int S_IDLE = 0, S_START = 1, S_NEWTON = 2;

struct Bucket {
    int L = 0, nb = 0;
    sphnse_plan* P = nullptr;
    long off = 0;              // first complex entry of the bucket in the concatenated vectors
    float *bsyn = nullptr, *gsyn = nullptr, *gsyn_r = nullptr, *gana_r = nullptr, *gana = nullptr, *hana = nullptr;
    size_t sb = 0, sg = 0, sa = 0, sh = 0;   // per-instance strides (floats)
    int* items = nullptr;
    int* item_off = nullptr;
    int ncta = 0;
    double* nu_dev = nullptr;
    TcBatch tcb;               // BF16X3: instance groups of the tensor-core synthesis
    TcBatchA tca;              //         and slots of the tensor-core analysis
    bool tc = false;
};

}  // namespace
}  // namespace sph

using namespace sph;

struct sphnse_ensemble {
    int n = 0;
    double Omega = 0;
    double rtol = 1e-6, atol = 1e-12, h_max = 1.0;
    int max_order = 5, newton_max = 4;
    int precision = SPHNSE_FP32;     // FP32 streaming, or BF16X3 tensor-core synthesis (batched)
    cudaStream_t stream = nullptr;   // the ensemble's own stream: all work, capture and replay
    cudaStream_t user = nullptr;     // the caller's stream, joined by events at API boundaries
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<int> L;
    std::vector<double> nu;
    std::vector<Bucket> buckets;
    std::vector<int> bucket_of, slot_of;     // instance -> bucket, position in bucket
    std::vector<long> off;                    // instance -> offset in concatenated vectors
    std::vector<int> nco;
    long total = 0;
    double2 *alpha = nullptr, *dif = nullptr, *y0 = nullptr, *psi = nullptr, *d = nullptr, *ynew = nullptr,
            *F = nullptr;
    InstPar* d_par = nullptr;
    InstPar* par = nullptr;          // pinned host copy, uploaded before each launch
    int2* d_btab = nullptr;          // block table (instance, block of the instance)
    int nbt = 0;
    unsigned long long* d_norms = nullptr;
    unsigned long long* h_norms = nullptr;
    std::vector<Ctl> ctl;
    cudaGraphExec_t g_rhs_alpha = nullptr, g_round = nullptr;
    int max_n = 0;
    long rounds = 0;                 // graph launches of the last advance
};

namespace {

int batched_rhs(sphnse_ensemble* E, const double2* x, double2* F) {
    int rc;
    for (auto& B : E->buckets) {
        sphnse_plan* P = B.P;
        P->stream = E->stream;
        const double* xb = reinterpret_cast<const double*>(x + B.off);
        double* Fb = reinterpret_cast<double*>(F + B.off);
        if (B.tc) {
            // all instances of the bucket share every table tile of the synthesis
            if ((rc = launch_prep_tc_batch(P, B.tcb, xb))) return rc;
            if ((rc = launch_synthesis_tc_batch(P, B.tcb, B.gsyn, B.sg, 0))) return rc;
        } else {
            if ((rc = launch_prep32_batch(P, B.nb, xb, B.bsyn, B.sb))) return rc;
            if ((rc = launch_synthesis_stream_batch(P, B.items, B.item_off, B.ncta, B.bsyn, B.sb, B.gsyn, B.sg, 0)))
                return rc;
        }
        if (ring4_ok(P)) {
            if ((rc = launch_ring4(P, B.nb, B.gsyn, B.sg, B.gana, B.sa, 0))) return rc;
        } else {
            if ((rc = launch_transpose(P, B.gsyn, B.gsyn_r, P->N + 1, P->nlat, 3 * B.nb, SPHNSE_FP32))) return rc;
            if ((rc = launch_ring_batch(P, B.nb, B.gsyn_r, B.sg, B.gana_r, B.sa))) return rc;
            if ((rc = launch_transpose(P, B.gana_r, B.gana, P->nlat, P->N + 1, 2 * B.nb, SPHNSE_FP32))) return rc;
        }
        if (B.tc) {
            if ((rc = launch_analysis_tc_batch(P, B.tca, B.gana, B.sa, B.hana, B.sh))) return rc;
        } else if ((rc = launch_analysis_stream_batch(P, B.items, B.item_off, B.ncta, B.gana, B.sa, B.hana, B.sh))) {
            return rc;
        }
        if ((rc = launch_finish32_batch(P, B.nb, B.hana, B.sh, xb, Fb, B.nu_dev))) return rc;
    }
    return SPHNSE_OK;
}

int upload_par(sphnse_ensemble* E) {
    return cudaMemcpyAsync(E->d_par, E->par, E->n * sizeof(InstPar), cudaMemcpyHostToDevice, E->stream) ==
                   cudaSuccess
               ? SPHNSE_OK
               : SPHNSE_E_CUDA;
}

int read_all_norms(sphnse_ensemble* E) {
    if (cudaMemcpyAsync(E->h_norms, E->d_norms, size_t(E->n) * 8 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, E->stream) != cudaSuccess ||
        cudaStreamSynchronize(E->stream) != cudaSuccess)
        return SPHNSE_E_CUDA;
    return SPHNSE_OK;
}

double nrm(const sphnse_ensemble* E, int i, int slot) {
    double v;
    std::memcpy(&v, &E->h_norms[size_t(i) * 8 + slot], sizeof(v));
    return v;
}

// capture a stream sequence into an executable graph
template <typename Fn>
int capture(sphnse_ensemble* E, cudaGraphExec_t* exec, Fn&& fn) {
    if (*exec) return SPHNSE_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(E->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) return SPHNSE_E_CUDA;
    const int rc = fn();
    const cudaError_t ce = cudaStreamEndCapture(E->stream, &g);
    if (rc) return rc;
    if (ce != cudaSuccess || !g) return SPHNSE_E_CUDA;
    const cudaError_t ie = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return ie == cudaSuccess ? SPHNSE_OK : SPHNSE_E_CUDA;
}

void destroy_ens(sphnse_ensemble* E) {
    if (!E) return;
    if (E->stream) cudaStreamSynchronize(E->stream);
    else cudaDeviceSynchronize();
    if (E->g_rhs_alpha) cudaGraphExecDestroy(E->g_rhs_alpha);
    if (E->g_round) cudaGraphExecDestroy(E->g_round);
    if (E->par) cudaFreeHost(E->par);
    if (E->d_btab) cudaFree(E->d_btab);
    if (E->ev_in) cudaEventDestroy(E->ev_in);
    if (E->ev_out) cudaEventDestroy(E->ev_out);
    for (auto& B : E->buckets) {
        void* ptrs[] = {B.bsyn, B.gsyn, B.gsyn_r, B.gana_r, B.gana, B.hana, B.items, B.item_off, B.nu_dev};
        for (void* q : ptrs)
            if (q) cudaFree(q);
        tc_batch_free(&B.tcb);
        tc_batch_ana_free(&B.tca);
        if (B.P) sphnse_plan_destroy(B.P);
    }
    void* ptrs[] = {E->alpha, E->dif, E->y0, E->psi, E->d, E->ynew, E->F, E->d_par, E->d_norms};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (E->h_norms) cudaFreeHost(E->h_norms);
    if (E->stream) cudaStreamDestroy(E->stream);
    delete E;
}

// order the ensemble's stream after the caller's work, and the caller's
// stream after the ensemble's work
void enter(sphnse_ensemble* E) {
    cudaEventRecord(E->ev_in, E->user);
    cudaStreamWaitEvent(E->stream, E->ev_in, 0);
}
int leave(sphnse_ensemble* E, int rc) {
    cudaEventRecord(E->ev_out, E->stream);
    cudaStreamWaitEvent(E->user, E->ev_out, 0);
    return rc;
}

int smallest_grid(int L) {
    // smallest even M = 2^a 3^b >= 3L + 2
    int best = 0;
    for (long a = 2; a <= 4096; a *= 2)
        for (long m = a; m <= 4096; m *= 3)
            if (m >= 3 * L + 2 && m % 2 == 0 && (best == 0 || m < best)) best = int(m);
    return best;
}

}  // namespace

extern "C" {

sphnse_ensemble* sphnse_ensemble_create(int n, const int* Ls, const double* nus, double Omega) {
    if (n < 1 || !Ls || !nus || !std::isfinite(Omega)) return nullptr;
    sphnse_ensemble* E = new (std::nothrow) sphnse_ensemble();
    if (!E) return nullptr;
    E->n = n;
    E->Omega = Omega;
    E->L.assign(Ls, Ls + n);
    E->nu.assign(nus, nus + n);
    std::map<int, std::vector<int>> byL;
    for (int i = 0; i < n; ++i) {
        if (Ls[i] < 1 || !(nus[i] >= 0.0)) {
            destroy_ens(E);
            return nullptr;
        }
        byL[Ls[i]].push_back(i);
    }
    E->bucket_of.resize(n);
    E->slot_of.resize(n);
    E->off.resize(n);
    E->nco.resize(n);
    long total = 0;
    int rc = SPHNSE_OK;
    for (auto& kv : byL) {
        Bucket B;
        B.L = kv.first;
        B.nb = int(kv.second.size());
        const int M = smallest_grid(B.L);
        B.P = M ? sphnse_plan_create(B.L, M / 2, M, 0.0, Omega) : nullptr;
        if (!B.P || sphnse_plan_set(B.P, SPHNSE_KEY_PRECISION, SPHNSE_FP32) != SPHNSE_OK) {
            if (B.P) sphnse_plan_destroy(B.P);
            destroy_ens(E);
            return nullptr;
        }
        const sphnse_plan* P = B.P;
        B.off = total;
        std::vector<double> nub;
        for (int s = 0; s < B.nb; ++s) {
            const int i = kv.second[s];
            E->bucket_of[i] = int(E->buckets.size());
            E->slot_of[i] = s;
            E->off[i] = total;
            E->nco[i] = P->n_coeff;
            total += P->n_coeff;
            nub.push_back(nus[i]);
        }
        const size_t g1 = size_t(P->N + 1) * P->nlat * 2;  // floats in one complex field
        B.sb = size_t(P->n_ext) * 6;
        B.sg = 3 * g1;
        B.sa = 2 * g1;
        B.sh = size_t(P->n_ext) * 4;
        auto fal = [&](float** q, size_t cnt) {
            if (!rc && cudaMalloc(reinterpret_cast<void**>(q), cnt * sizeof(float)) != cudaSuccess) rc = SPHNSE_E_NOMEM;
        };
        fal(&B.bsyn, B.sb * B.nb);
        fal(&B.gsyn, B.sg * B.nb);
        fal(&B.gsyn_r, B.sg * B.nb);
        fal(&B.gana_r, B.sa * B.nb);
        fal(&B.gana, B.sa * B.nb);
        fal(&B.hana, B.sh * B.nb);
        // LPT over (instance, m) items; costs L + 2 - m; instances interleaved so
        // that the same order of different instances streams at the same time
        std::vector<std::pair<int, int>> items;  // (cost, value)
        for (int m = 0; m <= P->N; ++m)
            for (int s = 0; s < B.nb; ++s) items.push_back({P->N + 2 - m, s * (P->N + 1) + m});
        const int G = std::min<int>(P->n_cta, int(items.size()));
        std::vector<std::vector<int>> bins(G);
        std::vector<long> load(G, 0);
        for (auto& it : items) {
            const int b = int(std::min_element(load.begin(), load.end()) - load.begin());
            bins[b].push_back(it.second);
            load[b] += it.first;
        }
        std::vector<int> flat, offs(1, 0);
        for (auto& bi : bins) {
            flat.insert(flat.end(), bi.begin(), bi.end());
            offs.push_back(int(flat.size()));
        }
        if (!rc && (cudaMalloc(reinterpret_cast<void**>(&B.items), flat.size() * sizeof(int)) != cudaSuccess ||
                    cudaMalloc(reinterpret_cast<void**>(&B.item_off), offs.size() * sizeof(int)) != cudaSuccess ||
                    cudaMalloc(reinterpret_cast<void**>(&B.nu_dev), B.nb * sizeof(double)) != cudaSuccess))
            rc = SPHNSE_E_NOMEM;
        if (!rc) {
            cudaMemcpy(B.items, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice);
            cudaMemcpy(B.item_off, offs.data(), offs.size() * sizeof(int), cudaMemcpyHostToDevice);
            cudaMemcpy(B.nu_dev, nub.data(), B.nb * sizeof(double), cudaMemcpyHostToDevice);
        }
        B.ncta = G;
        E->buckets.push_back(B);
        if (rc) {
            destroy_ens(E);
            return nullptr;
        }
    }
    E->total = total;
    for (int i = 0; i < n; ++i) E->max_n = std::max(E->max_n, E->nco[i]);
    auto al = [&](double2** q, size_t cnt) {
        if (!rc && cudaMalloc(reinterpret_cast<void**>(q), cnt * sizeof(double2)) != cudaSuccess) rc = SPHNSE_E_NOMEM;
        if (!rc) cudaMemset(*q, 0, cnt * sizeof(double2));
    };
    al(&E->alpha, total);
    al(&E->dif, 7 * size_t(total));
    al(&E->y0, total);
    al(&E->psi, total);
    al(&E->d, total);
    al(&E->ynew, total);
    al(&E->F, total);
    if (!rc && cudaMalloc(reinterpret_cast<void**>(&E->d_par), n * sizeof(InstPar)) != cudaSuccess) rc = SPHNSE_E_NOMEM;
    if (!rc && cudaMalloc(reinterpret_cast<void**>(&E->d_norms), size_t(n) * 8 * sizeof(unsigned long long)) != cudaSuccess)
        rc = SPHNSE_E_NOMEM;
    if (!rc && cudaMallocHost(reinterpret_cast<void**>(&E->h_norms), size_t(n) * 8 * sizeof(unsigned long long)) !=
                   cudaSuccess)
        rc = SPHNSE_E_NOMEM;
    if (!rc && cudaMallocHost(reinterpret_cast<void**>(&E->par), size_t(n) * sizeof(InstPar)) != cudaSuccess)
        rc = SPHNSE_E_NOMEM;
    if (!rc) {
        std::vector<int2> bt;
        for (int i = 0; i < n; ++i)
            for (int b = 0; b < (E->nco[i] + EB - 1) / EB; ++b) bt.push_back(make_int2(i, b));
        E->nbt = int(bt.size());
        if (cudaMalloc(reinterpret_cast<void**>(&E->d_btab), bt.size() * sizeof(int2)) != cudaSuccess)
            rc = SPHNSE_E_NOMEM;
        else
            cudaMemcpy(E->d_btab, bt.data(), bt.size() * sizeof(int2), cudaMemcpyHostToDevice);
    }
    if (rc) {
        destroy_ens(E);
        return nullptr;
    }
    if (cudaStreamCreateWithFlags(&E->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&E->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&E->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        destroy_ens(E);
        return nullptr;
    }
    for (auto& B : E->buckets) B.P->stream = E->stream;
    E->ctl.resize(n);
    for (int i = 0; i < n; ++i) {
        InstPar& p = E->par[i];
        std::memset(&p, 0, sizeof(p));
        p.off = E->off[i];
        p.n = E->nco[i];
        p.nu = E->nu[i];
        p.Omega = Omega;
        p.lm = E->buckets[E->bucket_of[i]].P->d_lm;
    }
    return E;
}

void sphnse_ensemble_destroy(sphnse_ensemble* E) { destroy_ens(E); }

int sphnse_ensemble_set_stream(sphnse_ensemble* E, void* stream) {
    if (!E) return SPHNSE_E_ARG;
    E->user = reinterpret_cast<cudaStream_t>(stream);
    return SPHNSE_OK;
}

// BF16X3: the buckets whose grids the tensor-core kernels support get their
// BF16 hi/lo tables, tensor maps and instance groups now (none of it may be
// allocated while a graph is being captured); the captured graphs are rebuilt.
static int set_precision(sphnse_ensemble* E, int prec) {
    if (prec != SPHNSE_FP32 && prec != SPHNSE_BF16X3) return SPHNSE_E_UNSUPPORTED;
    if (E->stream) cudaStreamSynchronize(E->stream);
    for (auto& B : E->buckets) {
        const bool want = prec == SPHNSE_BF16X3 && tc_supported(B.P);
        if (want && !B.tcb.btiles) {
            int rc = ensure_tables(B.P, SPHNSE_BF16X3);
            if (!rc) rc = tc_setup_synthesis(B.P);
            if (!rc) rc = tc_batch_init(B.P, B.nb, &B.tcb);
            if (!rc) rc = tc_batch_ana_init(B.P, B.nb, &B.tca);
            if (rc) return rc;
        }
        B.tc = want;
    }
    if (E->g_rhs_alpha) cudaGraphExecDestroy(E->g_rhs_alpha);
    if (E->g_round) cudaGraphExecDestroy(E->g_round);
    E->g_rhs_alpha = E->g_round = nullptr;
    E->precision = prec;
    return SPHNSE_OK;
}

int sphnse_ensemble_set(sphnse_ensemble* E, int key, double v) {
    if (!E || !std::isfinite(v)) return SPHNSE_E_ARG;
    switch (key) {
        case SPHNSE_KEY_RTOL: if (v <= 0) return SPHNSE_E_ARG; E->rtol = v; return SPHNSE_OK;
        case SPHNSE_KEY_ATOL: if (v <= 0) return SPHNSE_E_ARG; E->atol = v; return SPHNSE_OK;
        case SPHNSE_KEY_MAX_ORDER: if (v < 1 || v > SPHNSE_MAXK) return SPHNSE_E_ARG; E->max_order = int(v); return SPHNSE_OK;
        case SPHNSE_KEY_NEWTON_MAX_ITER: if (v < 1 || v > 1000) return SPHNSE_E_ARG; E->newton_max = int(v); return SPHNSE_OK;
        case SPHNSE_KEY_H_MAX: if (v <= 0) return SPHNSE_E_ARG; E->h_max = v; return SPHNSE_OK;
        case SPHNSE_KEY_PRECISION: return set_precision(E, int(v));
        default: return SPHNSE_E_ARG;
    }
}

int sphnse_ensemble_get(sphnse_ensemble* E, int key, double* v) {
    if (!E || !v) return SPHNSE_E_ARG;
    switch (key) {
        case SPHNSE_KEY_RTOL: *v = E->rtol; break;
        case SPHNSE_KEY_ATOL: *v = E->atol; break;
        case SPHNSE_KEY_MAX_ORDER: *v = E->max_order; break;
        case SPHNSE_KEY_NEWTON_MAX_ITER: *v = E->newton_max; break;
        case SPHNSE_KEY_H_MAX: *v = E->h_max; break;
        case SPHNSE_KEY_PRECISION: *v = E->precision; break;
        case SPHNSE_KEY_ROUNDS: *v = double(E->rounds); break;
        default: return SPHNSE_E_ARG;
    }
    return SPHNSE_OK;
}

int sphnse_ensemble_instance(sphnse_ensemble* E, int i, double** alpha, double** F, int* n_coeff) {
    if (!E || i < 0 || i >= E->n) return SPHNSE_E_ARG;
    if (alpha) *alpha = reinterpret_cast<double*>(E->alpha + E->off[i]);
    if (F) *F = reinterpret_cast<double*>(E->F + E->off[i]);
    if (n_coeff) *n_coeff = E->nco[i];
    return SPHNSE_OK;
}

static int ensemble_rhs_inner(sphnse_ensemble* E) {
    int rc = capture(E, &E->g_rhs_alpha, [&]() { return batched_rhs(E, E->alpha, E->F); });
    if (rc) return rc;
    return cudaGraphLaunch(E->g_rhs_alpha, E->stream) == cudaSuccess ? SPHNSE_OK : SPHNSE_E_CUDA;
}

int sphnse_ensemble_rhs(sphnse_ensemble* E) {
    if (!E) return SPHNSE_E_ARG;
    enter(E);
    return leave(E, ensemble_rhs_inner(E));
}

static int ensemble_init_inner(sphnse_ensemble* E, double t0) {
    int rc;
    if ((rc = ensemble_rhs_inner(E))) return rc;
    const double thr = E->atol / E->rtol;
    for (int i = 0; i < E->n; ++i) {
        E->par[i].flags = F_INIT;
        E->par[i].thr = thr;
    }
    if ((rc = upload_par(E))) return rc;
    cudaMemsetAsync(E->d_norms, 0, size_t(E->n) * 8 * sizeof(unsigned long long), E->stream);
    kb_wnorm<<<E->nbt, EB, 0, E->stream>>>(E->d_btab, E->d_par, F_INIT, E->F, E->alpha, E->d_norms, 0);
    if ((rc = read_all_norms(E))) return rc;
    for (int i = 0; i < E->n; ++i) {
        if (E->h_norms[size_t(i) * 8 + 7]) return SPHNSE_E_NONFINITE;
        const double rh = 1.25 * nrm(E, i, 0) / std::sqrt(E->rtol);
        const double h0 = rh > 0.0 ? std::min(E->h_max, 1.0 / rh) : E->h_max;
        Ctl& c = E->ctl[i];
        c = Ctl();
        c.t = t0;
        c.h = h0;
        c.h_dif = h0;
        c.k = 1;
        E->par[i].h0 = h0;
    }
    if ((rc = upload_par(E))) return rc;
    kb_init<<<E->nbt, EB, 0, E->stream>>>(E->d_btab, E->d_par, E->dif, E->F);
    return check_cuda(cudaGetLastError());
}

int sphnse_ensemble_init(sphnse_ensemble* E, double t0) {
    if (!E || !std::isfinite(t0)) return SPHNSE_E_ARG;
    enter(E);
    return leave(E, ensemble_init_inner(E, t0));
}

static int ensemble_advance_inner(sphnse_ensemble* E, int nsteps, sphnse_step_info* info);

int sphnse_ensemble_step(sphnse_ensemble* E, sphnse_step_info* info) {
    if (!E) return SPHNSE_E_ARG;
    enter(E);
    return leave(E, ensemble_advance_inner(E, 1, info));
}

int sphnse_ensemble_advance(sphnse_ensemble* E, int nsteps, sphnse_step_info* info) {
    if (!E || nsteps < 0) return SPHNSE_E_ARG;
    enter(E);
    return leave(E, ensemble_advance_inner(E, nsteps, info));
}

static int ensemble_advance_inner(sphnse_ensemble* E, int nsteps, sphnse_step_info* info) {
    const int n = E->n;
    double gam[SPHNSE_MAXK], iga[SPHNSE_MAXK], ec[SPHNSE_MAXK];
    {
        double g = 0.0;
        for (int k = 1; k <= SPHNSE_MAXK; ++k) {
            g += 1.0 / k;
            gam[k - 1] = g;
            iga[k - 1] = 1.0 / (g * (1.0 - KAPPA_E[k - 1]));
            ec[k - 1] = KAPPA_E[k - 1] * g + 1.0 / (k + 1.0);
        }
    }
    const double thr = E->atol / E->rtol;
    const int maxit = E->newton_max;
    const size_t nb = size_t(n) * 8 * sizeof(unsigned long long);
    int rc;
    // one round: accept / rescale / predict where flagged, the batched RHS at
    // ynew, the Newton update where flagged, and the norms to the host
    rc = capture(E, &E->g_round, [&]() {
        cudaStream_t st = E->stream;
        if (cudaMemsetAsync(E->d_norms, 0, nb, st) != cudaSuccess) return SPHNSE_E_CUDA;
        kb_accept<<<E->nbt, EB, 0, st>>>(E->d_btab, E->d_par, E->dif, E->d, E->alpha, E->ynew);
        kb_rescale<<<E->nbt, EB, 0, st>>>(E->d_btab, E->d_par, E->dif);
        kb_predict<<<E->nbt, EB, 0, st>>>(E->d_btab, E->d_par, E->alpha, E->dif, E->y0, E->psi, E->d, E->ynew,
                                           E->d_norms);
        int r = batched_rhs(E, E->ynew, E->F);
        if (r) return r;
        kb_newton<<<E->nbt, EB, 0, st>>>(E->d_btab, E->d_par, E->F, E->alpha, E->y0, E->psi, E->d, E->ynew,
                                          E->dif, E->d_norms);
        if (cudaMemcpyAsync(E->h_norms, E->d_norms, nb, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return SPHNSE_E_CUDA;
        return check_cuda(cudaGetLastError());
    });
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        Ctl& c = E->ctl[i];
        c.state = nsteps > 0 ? S_START : S_IDLE;
        c.steps_left = nsteps;
        c.attempts = 0;
        c.nofailed = true;
        c.pending_accept = false;
        c.rejections = 0;
        c.newton = 0;
        c.h_dif_before = c.h_dif;
    }
    E->rounds = 0;
    for (;;) {
        bool newton = false, accept = false;
        for (int i = 0; i < n; ++i) {
            Ctl& c = E->ctl[i];
            InstPar& p = E->par[i];
            p.flags = 0;
            if (c.pending_accept) {
                p.flags |= F_ACCEPT;
                p.ka = c.acc_k;
                c.pending_accept = false;
                accept = true;
            }
            if (c.state == S_START) {
                if (++c.attempts > 200) return SPHNSE_E_STEP_TOO_SMALL;
                c.hmin = 16.0 * EPS * std::fabs(c.t);
                const double h = std::min(E->h_max, std::max(c.hmin, c.h));
                c.h = h;
                const int k = c.k;
                if (h != c.h_dif) {
                    rescale_mat(k, h / c.h_dif, p.A);
                    p.flags |= F_RESCALE;
                    c.h_dif = h;
                    c.nconhk = 0;
                }
                if (h != c.miter_h || k != c.miter_k) {
                    c.havrate = 0;
                    c.miter_h = h;
                    c.miter_k = k;
                }
                c.ha = h;
                c.ka = k;
                p.k = k;
                p.c = h * iga[k - 1];
                p.thr = thr;
                for (int j = 0; j < SPHNSE_MAXK; ++j) p.g[j] = j < k ? gam[j] * iga[k - 1] : 0.0;
                p.flags |= F_PREDICT | F_NEWTON;
                c.state = S_NEWTON;
                c.it = 0;
                c.its = 0;
                c.oldnrm = 0.0;
                c.conv = false;
            } else if (c.state == S_NEWTON) {
                p.flags |= F_NEWTON;
            }
            newton = newton || (p.flags & F_NEWTON);
        }
        if (!newton) {
            // only the accepts of the last round remain
            if (accept) {
                if ((rc = upload_par(E))) return rc;
                kb_accept<<<E->nbt, EB, 0, E->stream>>>(E->d_btab, E->d_par, E->dif, E->d, E->alpha, E->ynew);
                if ((rc = check_cuda(cudaGetLastError()))) return rc;
            }
            break;
        }
        if ((rc = upload_par(E))) return rc;
        if (cudaGraphLaunch(E->g_round, E->stream) != cudaSuccess || cudaStreamSynchronize(E->stream) != cudaSuccess)
            return SPHNSE_E_CUDA;
        ++E->rounds;
        for (int i = 0; i < n; ++i) {
            Ctl& c = E->ctl[i];
            if (!(E->par[i].flags & F_NEWTON)) continue;
            if (E->h_norms[size_t(i) * 8 + 7]) return SPHNSE_E_NONFINITE;
            const int it = c.it;
            if (it == 0) c.ynorm = nrm(E, i, 4);
            for (int q = 0; q < 4; ++q) c.nrm[q] = nrm(E, i, q);
            c.its = it + 1;
            // the corrector's rate test (as sphnse_step)
            const double newnrm = c.nrm[0], minnrm = 100.0 * EPS * c.ynorm;
            bool stop = false, conv = false;
            if (newnrm <= minnrm) {
                stop = conv = true;
            } else if (it == 0) {
                if (c.havrate) {
                    const double errit = newnrm * c.rate / (1.0 - c.rate);
                    if (errit <= 0.05 * E->rtol) stop = conv = true;
                } else {
                    c.rate = 0.0;
                }
            } else if (newnrm > 0.9 * c.oldnrm) {
                stop = true;
            } else {
                c.rate = std::max(0.9 * c.rate, newnrm / c.oldnrm);
                c.havrate = 1;
                const double errit = newnrm * c.rate / (1.0 - c.rate);
                if (errit <= 0.5 * E->rtol) stop = conv = true;
                else if (it == maxit - 1) stop = true;
                else if (0.5 * E->rtol < errit * std::pow(c.rate, maxit - 1 - it)) stop = true;
            }
            c.oldnrm = newnrm;
            if (!stop && it + 1 < maxit) {
                c.it = it + 1;
                continue;
            }
            // the attempt is over
            c.newton += c.its;
            const double h = c.ha;
            const int k = c.ka;
            c.state = S_START;
            if (!conv) {
                ++c.rejections;
                if (h <= c.hmin) return SPHNSE_E_STEP_TOO_SMALL;
                c.h = std::max(c.hmin, 0.3 * h);
                continue;
            }
            const double err = c.nrm[1] * ec[k - 1];
            if (err > E->rtol) {
                ++c.rejections;
                if (h <= c.hmin) return SPHNSE_E_STEP_TOO_SMALL;
                if (c.nofailed) {
                    c.nofailed = false;
                    double hopt = h * std::max(0.1, 0.833 * std::pow(E->rtol / err, 1.0 / (k + 1)));
                    if (k > 1) {
                        const double errkm1 = c.nrm[2] * ec[k - 2];
                        const double hkm1 = h * std::max(0.1, 0.769 * std::pow(E->rtol / errkm1, 1.0 / k));
                        if (hkm1 > hopt) {
                            hopt = std::min(h, hkm1);
                            c.k = k - 1;
                        }
                    }
                    c.h = std::max(c.hmin, hopt);
                } else {
                    c.h = std::max(c.hmin, 0.5 * h);
                }
                continue;
            }
            // accepted: the differences are updated at the start of the next launch
            c.pending_accept = true;
            c.acc_k = k;
            c.t += h;
            c.nconhk = std::min(c.nconhk + 1, SPHNSE_MAXK + 2);
            if (c.nconhk >= k + 2) {
                double temp = 1.2 * std::pow(err / E->rtol, 1.0 / (k + 1));
                double hopt = temp > 0.1 ? h / temp : 10.0 * h;
                int kopt = k;
                if (k > 1) {
                    const double errkm1 = c.nrm[2] * ec[k - 2];
                    temp = 1.3 * std::pow(errkm1 / E->rtol, 1.0 / k);
                    const double hkm1 = temp > 0.1 ? h / temp : 10.0 * h;
                    if (hkm1 > hopt) {
                        hopt = hkm1;
                        kopt = k - 1;
                    }
                }
                if (k < E->max_order) {
                    const double errkp1 = c.nrm[3] * ec[k];
                    temp = 1.4 * std::pow(errkp1 / E->rtol, 1.0 / (k + 2));
                    const double hkp1 = temp > 0.1 ? h / temp : 10.0 * h;
                    if (hkp1 > hopt) {
                        hopt = hkp1;
                        kopt = k + 1;
                    }
                }
                if (hopt > h) {
                    c.h = hopt;
                    if (kopt != k) {
                        c.k = kopt;
                        c.nconhk = 0;
                    }
                }
            }
            if (info) {
                sphnse_step_info& o = info[i];
                o.t = c.t;
                o.h = h;
                o.err = err;
                o.order = k;
                o.newton_iters = c.newton;
                o.rejections = c.rejections;
                o.rhs_evals = c.newton;
                o.next_order = c.k;
                o.next_h = c.h;
                o.h_dif_before = c.h_dif_before;
            }
            c.nofailed = true;
            c.attempts = 0;
            c.h_dif_before = c.h_dif;
            if (--c.steps_left == 0) c.state = S_IDLE;
        }
    }
    return SPHNSE_OK;
}

}  // extern "C"
