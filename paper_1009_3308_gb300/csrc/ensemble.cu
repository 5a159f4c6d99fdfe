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
// a controller kernel (one thread per instance; the same host/device
// functions as sphnse_step) that reads the instance's norms and sets its
// flags for the next round.  The rounds are a WHILE node of one graph launch
// per call, so the host waits once per call.  An instance that converges,
// rejects or accepts starts its next attempt in the next round, so no
// instance waits for another's rejected attempts or extra Newton iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "internal.h"
#include "controller.cuh"
#include "dmath.cuh"
#include "ndf_entry.cuh"
#include "newton.cuh"
#include "reduce.cuh"

namespace sph {
namespace {


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
    if (i < p.n) r[0] = wnorm_entry(v[o + i], y[o + i], p.thr);
    const int id[1] = {slot};
    block_amax<1>(norms + 8 * bt.x, r, id);
}

__global__ void kb_init(const int2* btab, const InstPar* par, double2* dif, const double2* F) {
    INST_PROLOGUE(F_INIT)
    init_dif_entry(dif + 7 * o, F + o, p.h0, p.n, i);
}

__global__ void kb_rescale(const int2* btab, const InstPar* par, double2* dif) {
    INST_PROLOGUE(F_RESCALE)
    rescale_entry(dif + 7 * o, p.A, p.k, p.n, i);
}

__global__ void kb_predict(const int2* btab, const InstPar* par, const double2* y, const double2* dif, double2* y0,
                           double2* psi, double2* d, double2* ynew, unsigned long long* norms) {
    INST_PROLOGUE_ALL(F_PREDICT)
    float r[1] = {0.f};
    // slot 4: ||y / max(|y|, thr)||_inf (FP32, as the corrector's norms)
    if (i < p.n)
        r[0] = predict_entry(y + o, dif + 7 * o, p.g, p.k, y0 + o, psi + o, d + o, ynew + o,
                             fmaxf(float(p.thr), 1e-30f), p.n, i);
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
    accept_entry(dif + 7 * o, d + o, y + o, ynew + o, p.ka, p.n, i);
}

// Per-call inputs and results of the device round loop.
struct EnsLoop {
    double rtol, thr, h_max;
    int nsteps, maxk, newton_max;
    int status, rounds, max_rounds;
    int active;          // some instance has a Newton update next round (controller blocks)
    unsigned arrived;    // controller blocks done with the current round
};

// One block, a thread per instance (strided): open a call of nsteps steps.
__global__ void kb_call_begin(StepCtl* sc, InstPar* par, unsigned long long* norms, EnsLoop* L, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        StepCtl& S = sc[i];
        S.rtol = L->rtol;
        S.thr = L->thr;
        S.h_max = L->h_max;
        S.maxk = L->maxk;
        S.newton_max = L->newton_max;
        S.nsteps = L->nsteps;
        S.done = 0;
        S.attempt = 0;
        S.status = SPHNSE_OK;
        S.sum_newton = 0;
        S.sum_rejections = 0;
        S.accept = 0;
        S.phase = L->nsteps > 0 ? 1 : 0;
        par[i].flags = 0;
        for (int q = 0; q < 8; ++q) norms[8 * size_t(i) + q] = 0ull;
    }
    if (threadIdx.x == 0) {
        L->status = SPHNSE_OK;
        L->rounds = 0;
        L->active = 0;
        L->arrived = 0u;
    }
}

// A thread per instance, one warp per block (the controller is FP64 work, so
// it is spread over SMs): take the results of the round just run (Newton
// stopping rule; at the end of an attempt rejection or acceptance and the
// next order and step size), set each instance's flags and parameters for
// the next round and clear its norm slots.  The last block to finish
// continues the loop while some instance still has a Newton update to do.
// counted: this call ends a round (not the set-up call before the first).
constexpr int CTL_THREADS = 32;

__global__ void kb_round_ctl(StepCtl* sc, InstPar* par, unsigned long long* norms, sphnse_step_info* info,
                             EnsLoop* L, int n, int counted, cudaGraphConditionalHandle loop) {
    bool active = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        StepCtl& S = sc[i];
        InstPar& p = par[i];
        unsigned long long* nr = norms + 8 * size_t(i);
        if (p.flags & F_NEWTON) {
            double nv[5];
            for (int q = 0; q < 5; ++q) nv[q] = __longlong_as_double(static_cast<long long>(nr[q]));
            if (newton_control(S.nc, nv, nr[7] != 0ull)) {
                att_end(S);
                if (S.status != SPHNSE_OK) {
                    atomicCAS(&L->status, SPHNSE_OK, S.status);
                    S.phase = 0;
                } else {
                    if (S.accept) {
                        // the last accepted step, with the call's totals
                        sphnse_step_info& I = info[i];
                        fill_info(S, I);
                        I.newton_iters = I.rhs_evals = S.sum_newton;
                        I.rejections = S.sum_rejections;
                    }
                    S.phase = S.done < S.nsteps ? 1 : 0;
                }
            }
        }
        int flags = 0;
        if (S.accept) {
            flags |= F_ACCEPT;
            p.ka = S.k_acc;
            S.accept = 0;
        }
        if (S.phase == 1) {
            att_begin(S);
            if (S.do_rescale) {
                flags |= F_RESCALE;
                for (int q = 0; q < SPHNSE_MAXK * SPHNSE_MAXK; ++q) p.A[q] = S.A[q];
            }
            flags |= F_PREDICT | F_NEWTON;
            p.k = S.k;
            p.c = S.nc.c;
            p.thr = S.thr;
            for (int q = 0; q < SPHNSE_MAXK; ++q) p.g[q] = S.g[q];
            S.phase = 2;
        } else if (S.phase == 2) {
            flags |= F_NEWTON;
        }
        p.flags = flags;
        for (int q = 0; q < 8; ++q) nr[q] = 0ull;
        active = active || (flags & F_NEWTON);
    }
    active = __syncthreads_or(active);
    if (threadIdx.x != 0) return;
    if (active) atomicOr(&L->active, 1);
    __threadfence();
    if (atomicAdd(&L->arrived, 1u) != gridDim.x - 1) return;
    // the last block: every block's flags and errors are visible
    __threadfence();
    const bool any = atomicExch(&L->active, 0) != 0;
    L->arrived = 0u;
    if (counted) ++L->rounds;
    int status = atomicAdd(&L->status, 0);
    // every round advances a Newton iteration, an attempt or a step of each
    // active instance, so the loop ends by itself; the cap only guards
    // against a controller fault
    if (any && status == SPHNSE_OK && L->rounds >= L->max_rounds) status = L->status = SPHNSE_E_STEP_TOO_SMALL;
    cudaGraphSetConditional(loop, any && status == SPHNSE_OK ? 1u : 0u);
}

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
    double syn_us = 0;         // tuned synthesis duration (0: not tuned)
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
    StepCtl* d_sc = nullptr;         // per-instance controller state (device resident)
    EnsLoop* d_loop = nullptr;
    EnsLoop* h_loop = nullptr;       // pinned
    sphnse_step_info* d_info = nullptr;
    sphnse_step_info* h_info = nullptr;  // pinned
    cudaGraphExec_t g_rhs_alpha = nullptr, g_adv = nullptr;
    int max_n = 0;
    long rounds = 0;                 // rounds of the last advance
    bool inited = false;             // sphnse_ensemble_init has set the controllers up
    bool autotune = true;            // time the tensor-core synthesis shapes per bucket
    int syn_cluster = 1;             // without the autotuner: CTAs per cluster of the batched synthesis
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
    if (E->g_adv) cudaGraphExecDestroy(E->g_adv);
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
    void* ptrs[] = {E->alpha, E->dif, E->y0, E->psi, E->d, E->ynew, E->F, E->d_par, E->d_norms, E->d_sc,
                    E->d_loop, E->d_info};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    void* hptrs[] = {E->h_norms, E->h_loop, E->h_info};
    for (void* q : hptrs)
        if (q) cudaFreeHost(q);
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
    // smallest M = 2^a 3^b >= 3L + 2 (exact quadrature, Eq. (M_choice)) that
    // the batched FP32 streaming kernels take: M >= 128 and a multiple of 16,
    // i.e. nh = M / 4 northern latitudes, at least 32 and a multiple of 4.
    // A grid above 3L + 2 gives the same F (up to rounding).
    int best = 0;
    for (long a = 2; a <= 4096; a *= 2)
        for (long m = a; m <= 4096; m *= 3)
            if (m >= 3 * L + 2 && m >= 128 && m % 16 == 0 && (best == 0 || m < best)) best = int(m);
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
    if (!rc && (cudaMalloc(reinterpret_cast<void**>(&E->d_sc), size_t(n) * sizeof(StepCtl)) != cudaSuccess ||
                cudaMalloc(reinterpret_cast<void**>(&E->d_loop), sizeof(EnsLoop)) != cudaSuccess ||
                cudaMallocHost(reinterpret_cast<void**>(&E->h_loop), sizeof(EnsLoop)) != cudaSuccess ||
                cudaMalloc(reinterpret_cast<void**>(&E->d_info), size_t(n) * sizeof(sphnse_step_info)) != cudaSuccess ||
                cudaMallocHost(reinterpret_cast<void**>(&E->h_info), size_t(n) * sizeof(sphnse_step_info)) !=
                    cudaSuccess))
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
// Autotuner of the batched tensor-core synthesis of one bucket: every
// (instances per group, pipeline stages) shape that fits (group widths 1..9,
// stages 6, 5, 4) is built, its B tiles prepared from the current states and
// its synthesis timed with CUDA events (one warm-up, three timed launches on
// the ensemble's stream); the fastest is kept.  The shape changes neither the
// result of an instance's column nor the other stages.
static int tune_synthesis(sphnse_ensemble* E, Bucket& B) {
    sphnse_plan* P = B.P;
    const double* xb = reinterpret_cast<const double*>(E->alpha + B.off);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return SPHNSE_E_CUDA;
    }
    TcBatch best;
    float best_ms = 0.f;
    std::vector<std::array<int, 3>> seen;
    int rc = SPHNSE_OK;
    for (int cs = 1; cs <= 4 && !rc; cs *= 2)
        for (int ng = 1; ng <= std::min(B.nb, 9) && !rc; ++ng)
        for (int ns = 6; ns >= 4 && !rc; --ns) {
            TcBatch T;
            const int irc = tc_batch_init(P, B.nb, &T, ng, ns, cs);
            if (irc == SPHNSE_E_UNSUPPORTED) continue;   // no resident cluster of this shape
            if ((rc = irc)) break;
            const std::array<int, 3> shape{T.ng, T.ns, T.cs};
            if (T.ns < 4 || std::find(seen.begin(), seen.end(), shape) != seen.end()) {
                tc_batch_free(&T);
                continue;
            }
            seen.push_back(shape);
            float ms = 0.f;
            rc = launch_prep_tc_batch(P, T, xb);
            if (!rc) rc = launch_synthesis_tc_batch(P, T, B.gsyn, B.sg, 0);
            if (!rc && cudaEventRecord(e0, E->stream) != cudaSuccess) rc = SPHNSE_E_CUDA;
            for (int r = 0; r < 3 && !rc; ++r) rc = launch_synthesis_tc_batch(P, T, B.gsyn, B.sg, 0);
            if (!rc && (cudaEventRecord(e1, E->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = SPHNSE_E_CUDA;
            if (!rc && (!best.btiles || ms < best_ms)) {
                tc_batch_free(&best);
                best = T;
                best_ms = ms;
            } else {
                tc_batch_free(&T);
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc || !best.btiles) {
        tc_batch_free(&best);
        return rc ? rc : SPHNSE_E_UNSUPPORTED;
    }
    B.tcb = best;
    B.syn_us = 1e3 * best_ms / 3.0;
    return SPHNSE_OK;
}

static int set_precision(sphnse_ensemble* E, int prec) {
    if (prec != SPHNSE_FP32 && prec != SPHNSE_BF16X3) return SPHNSE_E_UNSUPPORTED;
    if (E->stream) cudaStreamSynchronize(E->stream);
    for (auto& B : E->buckets) {
        const bool want = prec == SPHNSE_BF16X3 && tc_supported(B.P);
        if (want && !B.tcb.btiles) {
            int rc = ensure_tables(B.P, SPHNSE_BF16X3);
            if (!rc) rc = tc_setup_synthesis(B.P);
            if (!rc) rc = E->autotune ? tune_synthesis(E, B) : tc_batch_init(B.P, B.nb, &B.tcb, 9, 6, E->syn_cluster);
            if (!rc) rc = tc_batch_ana_init(B.P, B.nb, &B.tca);
            if (rc) return rc;
        }
        B.tc = want;
    }
    if (E->g_rhs_alpha) cudaGraphExecDestroy(E->g_rhs_alpha);
    if (E->g_adv) cudaGraphExecDestroy(E->g_adv);
    E->g_rhs_alpha = E->g_adv = nullptr;
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
        case SPHNSE_KEY_AUTOTUNE: if (v != 0 && v != 1) return SPHNSE_E_ARG; E->autotune = v != 0; return SPHNSE_OK;
        case SPHNSE_KEY_SYN_CLUSTER:
            if (v != 1 && v != 2 && v != 4) return SPHNSE_E_ARG;
            E->syn_cluster = int(v);
            return SPHNSE_OK;
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
        case SPHNSE_KEY_AUTOTUNE: *v = E->autotune ? 1.0 : 0.0; break;
        case SPHNSE_KEY_BUCKETS: *v = double(E->buckets.size()); break;
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

int sphnse_ensemble_bucket(sphnse_ensemble* E, int b, int* L, int* count, int* group, int* stages, int* cluster,
                           double* syn_us) {
    if (!E || b < 0 || b >= int(E->buckets.size())) return SPHNSE_E_ARG;
    const Bucket& B = E->buckets[size_t(b)];
    if (L) *L = B.L;
    if (count) *count = B.nb;
    if (group) *group = B.tc ? B.tcb.ng : 0;
    if (stages) *stages = B.tc ? B.tcb.ns : 0;
    if (cluster) *cluster = B.tc ? B.tcb.cs : 0;
    if (syn_us) *syn_us = B.tc ? B.syn_us : 0.0;
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
    std::vector<StepCtl> sc(E->n);
    for (int i = 0; i < E->n; ++i) {
        if (E->h_norms[size_t(i) * 8 + 7]) return SPHNSE_E_NONFINITE;
        const double rh = 1.25 * nrm(E, i, 0) / std::sqrt(E->rtol);
        const double h0 = rh > 0.0 ? std::min(E->h_max, 1.0 / rh) : E->h_max;
        StepCtl& S = sc[i];
        S = StepCtl{};
        ndf_constants(false, S.gamma, S.iga, S.ec);
        S.nu = E->nu[i];
        S.omega = E->Omega;
        S.t = t0;
        S.h = h0;
        S.t_end = INFINITY;
        S.h_dif = h0;
        S.order = 1;
        E->par[i].h0 = h0;
    }
    if ((rc = upload_par(E))) return rc;
    if (cudaMemcpyAsync(E->d_sc, sc.data(), sc.size() * sizeof(StepCtl), cudaMemcpyHostToDevice, E->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(E->stream) != cudaSuccess)
        return SPHNSE_E_CUDA;
    E->inited = true;
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

// The advance graph: open the call, set up the first round, then a WHILE node
// over rounds (accept / rescale / predictor where flagged, one batched RHS,
// the Newton update where flagged, the controller), then the last accepts.
static int build_advance_graph(sphnse_ensemble* E) {
    if (E->g_adv) return SPHNSE_OK;
    const cudaStream_t cs = E->stream;
    const int nctl = std::min(1024, (E->n + 31) / 32 * 32);
    const int nblk = (E->n + CTL_THREADS - 1) / CTL_THREADS;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle h;
    cudaGraph_t body = nullptr;
    int rc = SPHNSE_OK;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
              cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess &&
              cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess;
    if (ok) {
        kb_call_begin<<<1, nctl, 0, cs>>>(E->d_sc, E->d_par, E->d_norms, E->d_loop, E->n);
        kb_round_ctl<<<nblk, CTL_THREADS, 0, cs>>>(E->d_sc, E->d_par, E->d_norms, E->d_info, E->d_loop, E->n, 0, h);
        cudaStreamCaptureStatus status;
        cudaGraph_t capg = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        cudaGraphNodeParams cp = {};
        cudaGraphNode_t node;
        ok = cudaStreamGetCaptureInfo(cs, &status, nullptr, &capg, &deps, nullptr, &ndeps) == cudaSuccess &&
             status == cudaStreamCaptureStatusActive;
        if (ok) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            ok = cudaGraphAddNode(&node, capg, deps, nullptr, ndeps, &cp) == cudaSuccess &&
                 cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies) ==
                     cudaSuccess;
            if (ok) body = cp.conditional.phGraph_out[0];
        }
        kb_accept<<<E->nbt, EB, 0, cs>>>(E->d_btab, E->d_par, E->dif, E->d, E->alpha, E->ynew);
        cudaGraph_t out = nullptr;
        ok = cudaStreamEndCapture(cs, &out) == cudaSuccess && ok;
    }
    ok = ok && body && cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) ==
                           cudaSuccess;
    if (ok) {
        kb_accept<<<E->nbt, EB, 0, cs>>>(E->d_btab, E->d_par, E->dif, E->d, E->alpha, E->ynew);
        kb_rescale<<<E->nbt, EB, 0, cs>>>(E->d_btab, E->d_par, E->dif);
        kb_predict<<<E->nbt, EB, 0, cs>>>(E->d_btab, E->d_par, E->alpha, E->dif, E->y0, E->psi, E->d, E->ynew,
                                           E->d_norms);
        rc = batched_rhs(E, E->ynew, E->F);
        kb_newton<<<E->nbt, EB, 0, cs>>>(E->d_btab, E->d_par, E->F, E->alpha, E->y0, E->psi, E->d, E->ynew, E->dif,
                                          E->d_norms);
        kb_round_ctl<<<nblk, CTL_THREADS, 0, cs>>>(E->d_sc, E->d_par, E->d_norms, E->d_info, E->d_loop, E->n, 1, h);
        cudaGraph_t out = nullptr;
        ok = cudaStreamEndCapture(cs, &out) == cudaSuccess && ok && rc == SPHNSE_OK;
    }
    if (ok) ok = cudaGraphInstantiate(&E->g_adv, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (!ok) {
        E->g_adv = nullptr;
        return rc ? rc : SPHNSE_E_CUDA;
    }
    return SPHNSE_OK;
}

static int ensemble_advance_inner(sphnse_ensemble* E, int nsteps, sphnse_step_info* info) {
    if (!E->inited) return SPHNSE_E_ARG;
    int rc;
    if ((rc = build_advance_graph(E))) return rc;
    EnsLoop& L = *E->h_loop;
    L = EnsLoop{};
    L.rtol = E->rtol;
    L.thr = E->atol / E->rtol;
    L.h_max = E->h_max;
    L.nsteps = nsteps;
    L.maxk = E->max_order;
    L.newton_max = E->newton_max;
    L.max_rounds = int(std::min<long>(1L << 30, long(nsteps) * 200 * (E->newton_max + 1) + 16));
    const size_t ib = size_t(E->n) * sizeof(sphnse_step_info);
    if (cudaMemcpyAsync(E->d_loop, E->h_loop, sizeof(EnsLoop), cudaMemcpyHostToDevice, E->stream) != cudaSuccess ||
        cudaGraphLaunch(E->g_adv, E->stream) != cudaSuccess ||
        cudaMemcpyAsync(E->h_loop, E->d_loop, sizeof(EnsLoop), cudaMemcpyDeviceToHost, E->stream) != cudaSuccess ||
        (info && cudaMemcpyAsync(E->h_info, E->d_info, ib, cudaMemcpyDeviceToHost, E->stream) != cudaSuccess) ||
        cudaStreamSynchronize(E->stream) != cudaSuccess)
        return SPHNSE_E_CUDA;
    E->rounds = L.rounds;
    if (info && nsteps > 0) std::memcpy(info, E->h_info, ib);
    return L.status;
}

}  // extern "C"
