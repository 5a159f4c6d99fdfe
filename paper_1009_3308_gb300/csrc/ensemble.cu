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
// sphnse_step, Sec. 4.2 Eq. (ode_disc)).  The controllers run in lockstep by
// attempt and Newton iteration: per-instance parameters live in a device
// array read by the batched kernels, inactive instances are masked, and the
// host reads all instances' norms once per Newton iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "internal.h"
#include "reduce.cuh"

namespace sph {
namespace {

constexpr double EPS = 2.220446049250313e-16;
const double KAPPA_E[SPHNSE_MAXK] = {-0.1850, -1.0 / 9.0, -0.0823, -0.0415, 0.0};

struct InstPar {
    long off;      // offset (complex entries) of this instance in the concatenated vectors
    int n;         // packed entries
    int k;         // order of the current attempt
    int active;    // participates in the current launch
    int rescale;   // rescale the differences in this attempt
    double c;      // h * iga_k
    double nu, Omega, thr;
    const int2* lm;
    double g[SPHNSE_MAXK];
    double A[SPHNSE_MAXK * SPHNSE_MAXK];
    double h0;     // initial step (init kernel)
};

#define INST_PROLOGUE                                        \
    const InstPar& p = par[blockIdx.y];                      \
    if (!p.active) return;                                   \
    const int i = blockIdx.x * blockDim.x + threadIdx.x;     \
    if (i >= p.n) return;                                    \
    const long o = p.off;

// the norm kernels keep every thread of an active block to the end (block reduction)
#define INST_PROLOGUE_ALL                                    \
    const InstPar& p = par[blockIdx.y];                      \
    if (!p.active) return;                                   \
    const int i = blockIdx.x * blockDim.x + threadIdx.x;     \
    const long o = p.off;

__global__ void kb_wnorm(const InstPar* par, const double2* v, const double2* y, unsigned long long* norms, int slot) {
    INST_PROLOGUE_ALL
    double r[1] = {0.0};
    if (i < p.n) {
        const double2 a = v[o + i], b = y[o + i];
        r[0] = fmax(fabs(a.x) / fmax(fabs(b.x), p.thr), fabs(a.y) / fmax(fabs(b.y), p.thr));
    }
    const int id[1] = {slot};
    block_amax<1>(norms + 8 * blockIdx.y, r, id);
}

__global__ void kb_init(const InstPar* par, double2* dif, const double2* F) {
    INST_PROLOGUE
    const double2 f = F[o + i];
    double2* D = dif + 7 * o;
    D[i] = make_double2(p.h0 * f.x, p.h0 * f.y);
    for (int j = 1; j < SPHNSE_MAXK + 2; ++j) D[size_t(j) * p.n + i] = make_double2(0.0, 0.0);
}

__global__ void kb_rescale(const InstPar* par, double2* dif) {
    INST_PROLOGUE
    if (!p.rescale) return;
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

__global__ void kb_predict(const InstPar* par, const double2* y, const double2* dif, double2* y0, double2* psi,
                           double2* d, double2* ynew) {
    INST_PROLOGUE
    const double2* D = dif + 7 * o;
    double2 a = y[o + i], q = make_double2(0.0, 0.0);
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
}

__global__ void kb_newton(const InstPar* par, const double2* F, const double2* y, const double2* y0,
                          const double2* psi, double2* d, double2* ynew, const double2* dif,
                          unsigned long long* norms) {
    INST_PROLOGUE_ALL
    double nv[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < p.n) {
        const int L = p.lm[i].x, m = p.lm[i].y;
        const double lam = double(L) * (L + 1.0);
        const double mr = 1.0 + p.c * p.nu * lam, mi = -p.c * 2.0 * p.Omega * m / lam;
        const double2 f = F[o + i], ps = psi[o + i], dd = d[o + i], yo = y[o + i], yn = ynew[o + i], a0 = y0[o + i];
        const double rx = p.c * f.x - (ps.x + dd.x), ry = p.c * f.y - (ps.y + dd.y);
        const double den = mr * mr + mi * mi;
        const double dlx = (rx * mr + ry * mi) / den, dly = (ry * mr - rx * mi) / den;
        const double thr = p.thr;
        const double wx = fmax(fmax(fabs(yo.x), fabs(yn.x)), thr), wy = fmax(fmax(fabs(yo.y), fabs(yn.y)), thr);
        nv[0] = fmax(fabs(dlx) / wx, fabs(dly) / wy);
        const double2 dn = make_double2(dd.x + dlx, dd.y + dly);
        const double2 yv = make_double2(a0.x + dn.x, a0.y + dn.y);
        d[o + i] = dn;
        ynew[o + i] = yv;
        const double vx = fmax(fmax(fabs(yo.x), fabs(yv.x)), thr), vy = fmax(fmax(fabs(yo.y), fabs(yv.y)), thr);
        nv[1] = fmax(fabs(dn.x) / vx, fabs(dn.y) / vy);
        const double2* D = dif + 7 * o;
        if (p.k >= 2) {
            const double2 q = D[size_t(p.k - 1) * p.n + i];
            nv[2] = fmax(fabs(q.x + dn.x) / vx, fabs(q.y + dn.y) / vy);
        }
        const double2 r2 = D[size_t(p.k) * p.n + i];
        nv[3] = fmax(fabs(dn.x - r2.x) / vx, fabs(dn.y - r2.y) / vy);
    }
    const int id[4] = {0, 1, 2, 3};
    block_amax<4>(norms + 8 * blockIdx.y, nv, id);
}

__global__ void kb_accept(const InstPar* par, double2* dif, const double2* d, double2* y, const double2* ynew) {
    INST_PROLOGUE
    double2* D = dif + 7 * o;
    const int k = p.k;
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
};

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
    std::vector<InstPar> par;
    unsigned long long* d_norms = nullptr;
    unsigned long long* h_norms = nullptr;
    std::vector<Ctl> ctl;
    cudaGraphExec_t g_rhs_alpha = nullptr, g_newton = nullptr;
    int max_n = 0;
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

dim3 egrid(const sphnse_ensemble* E) { return dim3((E->max_n + 255) / 256, E->n); }

int upload_par(sphnse_ensemble* E) {
    return cudaMemcpyAsync(E->d_par, E->par.data(), E->n * sizeof(InstPar), cudaMemcpyHostToDevice, E->stream) ==
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
    if (E->g_newton) cudaGraphExecDestroy(E->g_newton);
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
    E->par.resize(n);
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
    if (E->g_newton) cudaGraphExecDestroy(E->g_newton);
    E->g_rhs_alpha = E->g_newton = nullptr;
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
    for (auto& p : E->par) {
        p.active = 1;
        p.thr = thr;
    }
    if ((rc = upload_par(E))) return rc;
    cudaMemsetAsync(E->d_norms, 0, size_t(E->n) * 8 * sizeof(unsigned long long), E->stream);
    kb_wnorm<<<egrid(E), 256, 0, E->stream>>>(E->d_par, E->F, E->alpha, E->d_norms, 0);
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
    kb_init<<<egrid(E), 256, 0, E->stream>>>(E->d_par, E->dif, E->F);
    return check_cuda(cudaGetLastError());
}

int sphnse_ensemble_init(sphnse_ensemble* E, double t0) {
    if (!E || !std::isfinite(t0)) return SPHNSE_E_ARG;
    enter(E);
    return leave(E, ensemble_init_inner(E, t0));
}

static int ensemble_step_inner(sphnse_ensemble* E, sphnse_step_info* info);

int sphnse_ensemble_step(sphnse_ensemble* E, sphnse_step_info* info) {
    if (!E) return SPHNSE_E_ARG;
    enter(E);
    return leave(E, ensemble_step_inner(E, info));
}

static int ensemble_step_inner(sphnse_ensemble* E, sphnse_step_info* info) {
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
    int rc;
    for (auto& c : E->ctl) {
        c.done = false;
        c.nofailed = true;
        c.rejections = 0;
        c.newton = 0;
        c.h_dif_before = c.h_dif;
    }
    // Newton iteration graph: batched RHS of all instances at ynew + masked update
    rc = capture(E, &E->g_newton, [&]() {
        int r = batched_rhs(E, E->ynew, E->F);
        if (r) return r;
        kb_newton<<<egrid(E), 256, 0, E->stream>>>(E->d_par, E->F, E->alpha, E->y0, E->psi, E->d, E->ynew, E->dif,
                                                   E->d_norms);
        return check_cuda(cudaGetLastError());
    });
    if (rc) return rc;
    for (int attempt = 0; attempt < 200; ++attempt) {
        int pending = 0;
        for (int i = 0; i < n; ++i) {
            Ctl& c = E->ctl[i];
            InstPar& p = E->par[i];
            p.active = 0;
            p.rescale = 0;
            c.attempting = false;
            if (c.done) continue;
            ++pending;
            c.hmin = 16.0 * EPS * std::fabs(c.t);
            double h = std::min(E->h_max, std::max(c.hmin, c.h));
            c.h = h;
            const int k = c.k;
            if (h != c.h_dif) {
                rescale_mat(k, h / c.h_dif, p.A);
                p.rescale = 1;
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
            p.active = 1;
            c.attempting = true;
            c.in_newton = true;
            c.conv = false;
            c.its = 0;
            c.oldnrm = 0.0;
        }
        if (!pending) break;
        if ((rc = upload_par(E))) return rc;
        kb_rescale<<<egrid(E), 256, 0, E->stream>>>(E->d_par, E->dif);
        kb_predict<<<egrid(E), 256, 0, E->stream>>>(E->d_par, E->alpha, E->dif, E->y0, E->psi, E->d, E->ynew);
        cudaMemsetAsync(E->d_norms, 0, size_t(n) * 8 * sizeof(unsigned long long), E->stream);
        kb_wnorm<<<egrid(E), 256, 0, E->stream>>>(E->d_par, E->alpha, E->alpha, E->d_norms, 4);
        if ((rc = check_cuda(cudaGetLastError()))) return rc;
        for (int it = 0; it < maxit; ++it) {
            bool any = false;
            for (int i = 0; i < n; ++i) {
                E->par[i].active = E->ctl[i].attempting && E->ctl[i].in_newton;
                any = any || E->par[i].active;
            }
            if (!any) break;
            if ((rc = upload_par(E))) return rc;
            // slot 4 (the weight norm of alpha) is only read at it == 0
            if (it > 0) cudaMemsetAsync(E->d_norms, 0, size_t(n) * 8 * sizeof(unsigned long long), E->stream);
            if (cudaGraphLaunch(E->g_newton, E->stream) != cudaSuccess) return SPHNSE_E_CUDA;
            if ((rc = read_all_norms(E))) return rc;
            for (int i = 0; i < n; ++i) {
                Ctl& c = E->ctl[i];
                if (!E->par[i].active) continue;
                if (E->h_norms[size_t(i) * 8 + 7]) return SPHNSE_E_NONFINITE;
                if (it == 0) c.ynorm = nrm(E, i, 4);
                for (int q = 0; q < 4; ++q) c.nrm[q] = nrm(E, i, q);
                c.its = it + 1;
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
                if (stop) {
                    c.in_newton = false;
                    c.conv = conv;
                }
            }
        }
        // decisions
        bool any_accept = false;
        for (int i = 0; i < n; ++i) {
            Ctl& c = E->ctl[i];
            InstPar& p = E->par[i];
            p.active = 0;
            if (!c.attempting) continue;
            c.newton += c.its;
            const double h = c.ha;
            const int k = c.ka;
            if (!c.conv) {
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
            // accepted
            p.active = 1;
            p.k = k;
            any_accept = true;
            c.done = true;
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
        }
        if (any_accept) {
            if ((rc = upload_par(E))) return rc;
            kb_accept<<<egrid(E), 256, 0, E->stream>>>(E->d_par, E->dif, E->d, E->alpha, E->ynew);
            if ((rc = check_cuda(cudaGetLastError()))) return rc;
        }
    }
    for (const auto& c : E->ctl)
        if (!c.done) return SPHNSE_E_STEP_TOO_SMALL;
    return SPHNSE_OK;
}

}  // extern "C"
