// Plan lifecycle: validation, host FP64 precompute, device tables and
// workspaces, and the RHS pipelines built from the kernels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>
#include <unordered_set>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>

#include "internal.h"

namespace sph {

int check_cuda(cudaError_t e) { return e == cudaSuccess ? SPHNSE_OK : SPHNSE_E_CUDA; }

static void fold_stage_events(sphnse_plan* P) {
    cudaStreamSynchronize(P->stream);
    for (int s = 0; s < SPHNSE_NSTAGES; ++s) {
        for (int i = 0; i + 1 < P->ev_used[s]; i += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, P->ev[s][i], P->ev[s][i + 1]) == cudaSuccess) {
                P->stage_ms[s] += ms;
                P->stage_n[s] += 1;
            }
        }
        P->ev_used[s] = 0;
    }
}

static void record_stage_event(sphnse_plan* P, int stage) {
    auto& v = P->ev[stage];
    if (P->ev_used[stage] >= int(v.size())) {
        if (v.size() >= 1 << 16) fold_stage_events(P);  // bound the pool
        if (P->ev_used[stage] >= int(v.size())) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            v.push_back(e);
        }
    }
    cudaEventRecord(v[P->ev_used[stage]++], P->stream);
}

void stage_begin(sphnse_plan* P, int stage) {
    P->stage_rec[stage] = (P->timing & (1u << stage)) && P->stage_calls[stage] % P->timing_period == 0;
    if (P->stage_rec[stage]) record_stage_event(P, stage);
}
void stage_end(sphnse_plan* P, int stage) {
    if (!(P->timing & (1u << stage))) return;
    if (P->stage_rec[stage]) record_stage_event(P, stage);
    P->stage_rec[stage] = false;
    ++P->stage_calls[stage];
}

static void free_tables(Tables& t) {
    if (t.syn) cudaFree(t.syn);
    if (t.ana) cudaFree(t.ana);
    if (t.syn_lo) cudaFree(t.syn_lo);
    if (t.ana_lo) cudaFree(t.ana_lo);
    t = Tables();
}

// Analysis layout: block (m, parity) of rows r0..r0+nr-1 stored [nh][nr] at
// offset r0 * nh (same total size as the synthesis layout).
template <typename F>
static void for_each_block(int N, F&& f) {
    for (int m = 0; m <= N; ++m) {
        const int ne = ext_even(N, m), no = ext_odd(N, m), e0 = ext_off(N, m);
        f(e0, ne);
        if (no > 0) f(e0 + ne, no);
    }
}

template <typename T, typename Conv>
static int upload_pair(sphnse_plan* P, Tables& t, Conv conv, bool lo) {
    const size_t nh = P->nh, ne = P->n_ext;
    const size_t count = ne * nh;
    std::vector<T> syn(count), ana(count);
    const double* src = P->psyn_host.data();
    for (size_t i = 0; i < count; ++i) syn[i] = conv(src[i], lo);
    for_each_block(P->N, [&](int r0, int nr) {
        const size_t base = size_t(r0) * nh;
        for (int j = 0; j < nr; ++j)
            for (size_t p = 0; p < nh; ++p) ana[base + p * nr + j] = syn[base + size_t(j) * nh + p];
    });
    void** dsyn = lo ? &t.syn_lo : &t.syn;
    void** dana = lo ? &t.ana_lo : &t.ana;
    if (cudaMalloc(dsyn, count * sizeof(T)) != cudaSuccess) return SPHNSE_E_NOMEM;
    if (cudaMalloc(dana, count * sizeof(T)) != cudaSuccess) return SPHNSE_E_NOMEM;
    if (cudaMemcpy(*dsyn, syn.data(), count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return SPHNSE_E_CUDA;
    if (cudaMemcpy(*dana, ana.data(), count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return SPHNSE_E_CUDA;
    t.bytes += 2 * count * sizeof(T);
    return SPHNSE_OK;
}

int ensure_tables(sphnse_plan* P, int prec) {
    Tables& t = P->tab[prec];
    if (t.built) return SPHNSE_OK;
    int rc = SPHNSE_OK;
    if (prec == SPHNSE_FP64) {
        rc = upload_pair<double>(P, t, [](double v, bool) { return v; }, false);
    } else if (prec == SPHNSE_FP32) {
        rc = upload_pair<float>(P, t, [](double v, bool) { return float(v); }, false);
    } else {
        // BF16 hi + lo split: hi = bf16(v), lo = bf16(v - hi)
        auto conv = [](double v, bool lo) {
            __nv_bfloat16 hi = __float2bfloat16_rn(float(v));
            if (!lo) return hi;
            return __float2bfloat16_rn(float(v - double(__bfloat162float(hi))));
        };
        rc = upload_pair<__nv_bfloat16>(P, t, conv, false);
        if (rc == SPHNSE_OK) rc = upload_pair<__nv_bfloat16>(P, t, conv, true);
    }
    if (rc != SPHNSE_OK) {
        free_tables(t);
        return rc;
    }
    t.built = true;
    return SPHNSE_OK;
}

void allow_dynamic_smem(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> cap;
    std::lock_guard<std::mutex> lk(mu);
    size_t& c = cap[kernel];
    if (bytes > c && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)) ==
                         cudaSuccess)
        c = bytes;
}

void prefer_max_smem(const void* kernel) {
    static std::mutex mu;
    static std::unordered_set<const void*> done;
    std::lock_guard<std::mutex> lk(mu);
    if (done.insert(kernel).second)
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

int rhs_device(sphnse_plan* P, const double* alpha, const double* forcing, double* out) {
    const int prec = P->precision == SPHNSE_FP64 ? SPHNSE_FP64 : SPHNSE_FP32;
    int rc;
    const bool tc = P->precision == SPHNSE_BF16X3 && tc_supported(P);
    const bool ring4 = prec == SPHNSE_FP32 && ring4_ok(P);
    // the tensor-core synthesis writes the latitude-pair-major layout the
    // four-step ring kernel reads contiguously (its epilogue warps are off the
    // streaming path); the FP32 streaming synthesis keeps the order-major one
    const int pairs = ring4 && tc;
    if (tc) {
        if ((rc = launch_synthesis_tc(P, alpha, pairs))) return rc;   // builds its coefficient tiles
    } else {
        if ((rc = launch_prep(P, alpha, nullptr, prec))) return rc;
        if ((rc = launch_synthesis(P, 3, prec))) return rc;
    }
    if (ring4) {
        if ((rc = launch_ring4(P, 1, static_cast<const float*>(P->d_gsyn), 0, static_cast<float*>(P->d_gana), 0,
                               pairs)))
            return rc;
    } else {
        if ((rc = launch_transpose(P, P->d_gsyn, P->d_gsyn_r, P->N + 1, P->nlat, 3, prec))) return rc;
        if ((rc = launch_ring(P, RING_RHS, prec, nullptr, nullptr, nullptr, nullptr, nullptr))) return rc;
        if ((rc = launch_transpose(P, P->d_gana_r, P->d_gana, P->nlat, P->N + 1, 2, prec))) return rc;
    }
    if (tc) {
        // the finish step runs in the analysis epilogue where its shared
        // memory fits
        rc = launch_analysis_finish_tc(P, alpha, forcing, out);
        if (rc != SPHNSE_E_UNSUPPORTED) return rc;
    }
    if ((rc = tc ? launch_analysis_tc(P, 2) : launch_analysis(P, 2, prec))) return rc;
    return launch_finish(P, 0, prec, alpha, forcing, out);
}

// J(alpha)^T w = -nu lambda w - D_s ( A_u[-(zeta + f) xhat x V] + A_zeta[(xhat x u) . V] ),
// V = S_u(D_s^{-1} w): the transpose of the linearised product, with the
// synthesis transpose S^T = D_s A W^{-1} (A the weighted analysis).
int rhs_adjoint_device(sphnse_plan* P, const double* alpha, const double* w, double* out) {
    const int prec = P->precision == SPHNSE_FP64 ? SPHNSE_FP64 : SPHNSE_FP32;
    int rc;
    if ((rc = launch_prep(P, alpha, w, prec))) return rc;
    if ((rc = launch_synthesis(P, 5, prec))) return rc;
    if ((rc = launch_transpose(P, P->d_gsyn, P->d_gsyn_r, P->N + 1, P->nlat, 5, prec))) return rc;
    if ((rc = launch_ring(P, RING_ADJOINT, prec, nullptr, nullptr, nullptr, nullptr, nullptr))) return rc;
    if ((rc = launch_transpose(P, P->d_gana_r, P->d_gana, P->nlat, P->N + 1, 3, prec))) return rc;
    if ((rc = launch_analysis(P, 3, prec))) return rc;
    return launch_finish(P, 2, prec, w, nullptr, out);
}

}  // namespace sph

using namespace sph;

static thread_local int g_last_error = SPHNSE_OK;

static void destroy_plan(sphnse_plan* P) {
    if (!P) return;
    if (P->stream) cudaStreamSynchronize(P->stream);
    else cudaDeviceSynchronize();
    for (auto& t : P->tab) free_tables(t);
    tc_free(P);
    host_io_free(P);
    if (P->ng_exec) cudaGraphExecDestroy(P->ng_exec);
    if (P->d_ctl) cudaFree(P->d_ctl);
    if (P->h_ctl) cudaFreeHost(P->h_ctl);
    if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
    if (P->sg_exec) cudaGraphExecDestroy(P->sg_exec);
    if (P->d_step) cudaFree(P->d_step);
    if (P->h_step) cudaFreeHost(P->h_step);
    if (P->d_info) cudaFree(P->d_info);
    if (P->h_info) cudaFreeHost(P->h_info);
    void* ptrs[] = {P->d_items, P->d_item_off, P->d_status,
                    P->d_x, P->d_s, P->d_isin32, P->d_rw, P->d_tw, P->d_tw32, P->d_ftw, P->d_lm, P->d_finc, P->d_prepc, P->d_finc32, P->d_prepc32, P->d_bsyn,
                    P->d_gsyn, P->d_gana, P->d_hana, P->d_gsyn_r, P->d_gana_r, P->d_grid, P->d_theta, P->d_w, P->d_work, P->d_tmp, P->d_norms};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (P->h_norms) cudaFreeHost(P->h_norms);
    for (auto& v : P->ev)
        for (auto e : v) cudaEventDestroy(e);
    delete P;
}

template <typename T>
static int dalloc(T** p, size_t bytes) {
    return cudaMalloc(reinterpret_cast<void**>(p), bytes) == cudaSuccess ? SPHNSE_OK : SPHNSE_E_NOMEM;
}

extern "C" {

int sphnse_last_error(void) { return g_last_error; }

const char* sphnse_error_string(int code) {
    switch (code) {
        case SPHNSE_OK: return "ok";
        case SPHNSE_E_ARG: return "invalid argument";
        case SPHNSE_E_INEXACT: return "nlon < 3L+2: quadrature not exact on the Galerkin integrals";
        case SPHNSE_E_NOMEM: return "out of memory";
        case SPHNSE_E_CUDA: return "CUDA runtime error";
        case SPHNSE_E_NONFINITE: return "non-finite value";
        case SPHNSE_E_STEP_TOO_SMALL: return "step size below minimum";
        case SPHNSE_E_TIMEOUT: return "bounded device wait timed out";
        case SPHNSE_E_UNSUPPORTED: return "unsupported configuration";
        case SPHNSE_E_TOO_LARGE: return "size exceeds the fixed scratch of the allocation-free entry point";
        default: return "unknown status";
    }
}

sphnse_plan* sphnse_plan_create(int L, int nlat, int nlon, double nu, double Omega) {
    g_last_error = SPHNSE_OK;
    if (L < 1 || nlon < 2 || (nlon % 2) || nlat != nlon / 2 || !(nu >= 0.0) || !std::isfinite(nu) ||
        !std::isfinite(Omega)) {
        g_last_error = SPHNSE_E_ARG;
        return nullptr;
    }
    if (nlon < 3 * L + 2) {
        g_last_error = SPHNSE_E_INEXACT;
        return nullptr;
    }
    FFTPlan fft;
    // the ring kernel keeps at most 3 butterflies per thread with <= 256 threads
    if (!make_fft_plan(nlon, &fft) || nlon > 1536) {
        g_last_error = SPHNSE_E_UNSUPPORTED;
        return nullptr;
    }
    sphnse_plan* P = new (std::nothrow) sphnse_plan();
    if (!P) {
        g_last_error = SPHNSE_E_NOMEM;
        return nullptr;
    }
    P->N = L;
    P->nlat = nlat;
    P->nlon = nlon;
    P->nh = (nlat + 1) / 2;
    P->nu = nu;
    P->Omega = Omega;
    P->fft = fft;
    P->n_coeff = n_packed(L);
    P->n_ext = n_ext(L);
    cudaGetDevice(&P->device);
    int rc = SPHNSE_OK;
    try {
        P->theta.resize(nlat);
        P->x.resize(nlat);
        P->s.resize(nlat);
        P->w.resize(nlat);
        gauss_legendre(nlat, P->theta.data(), P->x.data(), P->s.data(), P->w.data());
        P->psyn_host.resize(size_t(P->n_ext) * P->nh);
        legendre_table_syn(L, P->nh, P->x.data(), P->s.data(), P->psyn_host.data());
    } catch (...) {
        rc = SPHNSE_E_NOMEM;
    }
    // device constants
    std::vector<double> rw(nlat), tw(2 * size_t(nlon));
    std::vector<float> tw32(2 * size_t(nlon));
    for (int p = 0; p < nlat; ++p) rw[p] = (2.0 * M_PI / nlon) * P->w[p] / P->s[p];
    for (int t = 0; t < nlon; ++t) {
        const double ang = 2.0 * M_PI * double(t) / double(nlon);
        tw[2 * t] = std::cos(ang);
        tw[2 * t + 1] = -std::sin(ang);
        tw32[2 * t] = float(tw[2 * t]);
        tw32[2 * t + 1] = float(tw[2 * t + 1]);
    }
    std::vector<int2> lm(P->n_coeff);
    std::vector<double4_32a> finc(P->n_coeff), prepc(P->n_ext);
    auto eps = [](int l, int m) {
        return l <= m ? 0.0 : std::sqrt((double(l) * l - double(m) * m) / (4.0 * l * l - 1.0));
    };
    for (int m = 0, i = 0; m <= L; ++m)
        for (int l = (m > 0 ? m : 1); l <= L; ++l) {
            lm[i] = make_int2(l, m);
            const double lam = double(l) * (l + 1.0), isl = 1.0 / std::sqrt(lam);
            finc[i] = make_double4_32a(isl, l * eps(l + 1, m) * isl, (l + 1) * eps(l, m) * isl, lam);
            ++i;
        }
    // prep: zeta set lam^{1/2} a_K, theta set lam^{-1/2} a_K, phi set
    // (K-1) eps_{K,m} lam_{K-1}^{-1/2} a_{K-1} - (K+2) eps_{K+1,m} lam_{K+1}^{-1/2} a_{K+1}
    for (int m = 0; m <= L; ++m) {
        const int lo = m > 0 ? m : 1;
        auto isl = [&](int k) { return (k < lo || k > L) ? 0.0 : 1.0 / std::sqrt(double(k) * (k + 1.0)); };
        for (int K = m; K <= L + 1; ++K) {
            const bool in = K >= lo && K <= L;
            prepc[ext_row(L, m, K)] = make_double4_32a(in ? std::sqrt(double(K) * (K + 1.0)) : 0.0, isl(K),
                                                   (K - 1) * eps(K, m) * isl(K - 1),
                                                   -(K + 2) * eps(K + 1, m) * isl(K + 1));
        }
    }
    const size_t nc = size_t(P->n_coeff);
    const size_t sz_g = size_t(nlat) * (L + 1) * 2 * sizeof(double);
    if (!rc) rc = dalloc(&P->d_x, nlat * sizeof(double));
    if (!rc) rc = dalloc(&P->d_s, nlat * sizeof(double));
    if (!rc) rc = dalloc(&P->d_isin32, nlat * sizeof(float));
    if (!rc) rc = dalloc(&P->d_rw, nlat * sizeof(double));
    if (!rc) rc = dalloc(&P->d_tw, tw.size() * sizeof(double));
    if (!rc) rc = dalloc(&P->d_tw32, tw32.size() * sizeof(float));
    const std::vector<float> ftw = ring4_twiddles(nlon);
    if (!rc && !ftw.empty()) rc = dalloc(&P->d_ftw, ftw.size() * sizeof(float));
    if (!rc) rc = dalloc(&P->d_lm, nc * sizeof(int2));
    if (!rc) rc = dalloc(&P->d_finc, nc * sizeof(double4_32a));
    if (!rc) rc = dalloc(&P->d_prepc, size_t(P->n_ext) * sizeof(double4_32a));
    if (!rc) rc = dalloc(&P->d_finc32, nc * sizeof(float4));
    if (!rc) rc = dalloc(&P->d_prepc32, size_t(P->n_ext) * sizeof(float4));
    if (!rc) rc = dalloc(&P->d_bsyn, size_t(P->n_ext) * 10 * sizeof(double));
    if (!rc) rc = dalloc(&P->d_gsyn, 5 * sz_g);
    if (!rc) rc = dalloc(&P->d_gana, 3 * sz_g);
    if (!rc) rc = dalloc(&P->d_hana, size_t(P->n_ext) * 6 * sizeof(double));
    if (!rc) rc = dalloc(&P->d_gsyn_r, 5 * sz_g);
    if (!rc) rc = dalloc(&P->d_gana_r, 3 * sz_g);
    if (!rc) rc = dalloc(&P->d_work, 16 * nc * 2 * sizeof(double));
    if (!rc) rc = dalloc(&P->d_tmp, 2 * nc * 2 * sizeof(double));
    if (!rc) rc = dalloc(&P->d_norms, 16 * sizeof(unsigned long long));
    if (!rc && cudaMallocHost(reinterpret_cast<void**>(&P->h_norms), 16 * sizeof(double)) != cudaSuccess)
        rc = SPHNSE_E_NOMEM;
    auto up = [&](void* d, const void* h, size_t b) {
        if (!rc && cudaMemcpy(d, h, b, cudaMemcpyHostToDevice) != cudaSuccess) rc = SPHNSE_E_CUDA;
    };
    up(P->d_x, P->x.data(), nlat * sizeof(double));
    up(P->d_s, P->s.data(), nlat * sizeof(double));
    {
        std::vector<float> isin(nlat);
        for (int p = 0; p < nlat; ++p) isin[p] = float(1.0 / P->s[p]);
        up(P->d_isin32, isin.data(), nlat * sizeof(float));
    }
    up(P->d_rw, rw.data(), nlat * sizeof(double));
    up(P->d_tw, tw.data(), tw.size() * sizeof(double));
    up(P->d_tw32, tw32.data(), tw32.size() * sizeof(float));
    if (!ftw.empty()) up(P->d_ftw, ftw.data(), ftw.size() * sizeof(float));
    up(P->d_lm, lm.data(), nc * sizeof(int2));
    up(P->d_finc, finc.data(), nc * sizeof(double4_32a));
    up(P->d_prepc, prepc.data(), size_t(P->n_ext) * sizeof(double4_32a));
    {
        std::vector<float4> f32(nc), p32(P->n_ext);
        for (size_t i = 0; i < nc; ++i)
            f32[i] = make_float4(float(finc[i].x), float(finc[i].y), float(finc[i].z), float(finc[i].w));
        for (size_t i = 0; i < size_t(P->n_ext); ++i)
            p32[i] = make_float4(float(prepc[i].x), float(prepc[i].y), float(prepc[i].z), float(prepc[i].w));
        up(P->d_finc32, f32.data(), nc * sizeof(float4));
        up(P->d_prepc32, p32.data(), size_t(P->n_ext) * sizeof(float4));
    }
    // LPT schedule of the orders m (cost L + 2 - m table rows) over one
    // persistent CTA per SM for the streaming Legendre kernels
    if (!rc) {
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device);
        if (nsm < 1) nsm = 1;
        P->nsm = nsm;
        const int G = nsm < L + 1 ? nsm : L + 1;
        std::vector<std::vector<int>> bins(G);
        std::vector<long> load(G, 0);
        for (int m = 0; m <= L; ++m) {  // costs decrease with m
            int b = 0;
            for (int k = 1; k < G; ++k)
                if (load[k] < load[b]) b = k;
            bins[b].push_back(m);
            load[b] += L + 2 - m;
        }
        std::vector<int> items, off(1, 0);
        for (auto& bi : bins) {
            items.insert(items.end(), bi.begin(), bi.end());
            off.push_back(int(items.size()));
        }
        P->n_cta = G;
        rc = dalloc(&P->d_items, items.size() * sizeof(int));
        if (!rc) rc = dalloc(&P->d_item_off, off.size() * sizeof(int));
        if (!rc) rc = dalloc(&P->d_status, sizeof(unsigned));
        up(P->d_items, items.data(), items.size() * sizeof(int));
        up(P->d_item_off, off.data(), off.size() * sizeof(int));
        if (!rc && cudaMemset(P->d_status, 0, sizeof(unsigned)) != cudaSuccess) rc = SPHNSE_E_CUDA;
    }
    if (!rc) rc = ensure_tables(P, SPHNSE_FP64);
    if (rc) {
        destroy_plan(P);
        g_last_error = rc;
        return nullptr;
    }
    return P;
}

void sphnse_plan_destroy(sphnse_plan* plan) { destroy_plan(plan); }

int sphnse_set_stream(sphnse_plan* P, void* stream) {
    if (!P) return SPHNSE_E_ARG;
    P->stream = reinterpret_cast<cudaStream_t>(stream);
    return SPHNSE_OK;
}

int sphnse_plan_set(sphnse_plan* P, int key, double v) {
    if (!P || !std::isfinite(v)) return SPHNSE_E_ARG;
    switch (key) {
        case SPHNSE_KEY_PRECISION: {
            const int pr = int(v);
            if (pr != SPHNSE_FP64 && pr != SPHNSE_FP32 && pr != SPHNSE_BF16X3) return SPHNSE_E_ARG;
            int rc = ensure_tables(P, pr);
            if (rc) return rc;
            if (pr == SPHNSE_BF16X3 && (rc = ensure_tables(P, SPHNSE_FP32))) return rc;
            P->precision = pr;
            return SPHNSE_OK;
        }
        case SPHNSE_KEY_NU: if (v < 0) return SPHNSE_E_ARG; P->nu = v; return SPHNSE_OK;
        case SPHNSE_KEY_OMEGA: P->Omega = v; return SPHNSE_OK;
        case SPHNSE_KEY_RTOL: if (v <= 0) return SPHNSE_E_ARG; P->rtol = v; return SPHNSE_OK;
        case SPHNSE_KEY_ATOL: if (v <= 0) return SPHNSE_E_ARG; P->atol = v; return SPHNSE_OK;
        case SPHNSE_KEY_MAX_ORDER: if (v < 1 || v > SPHNSE_MAXK) return SPHNSE_E_ARG; P->max_order = int(v); return SPHNSE_OK;
        case SPHNSE_KEY_NEWTON_MAX_ITER: if (v < 1 || v > 1000) return SPHNSE_E_ARG; P->newton_max = int(v); return SPHNSE_OK;
        case SPHNSE_KEY_H_MAX: if (v <= 0) return SPHNSE_E_ARG; P->h_max = v; return SPHNSE_OK;
        case SPHNSE_KEY_BDF: P->bdf = v != 0.0; return SPHNSE_OK;
        case SPHNSE_KEY_CORIOLIS_SPLIT: P->coriolis_split = v != 0.0; return SPHNSE_OK;
        case SPHNSE_KEY_TIMING_PERIOD: if (v < 1 || v > 1e6) return SPHNSE_E_ARG; P->timing_period = int(v); return SPHNSE_OK;
        case SPHNSE_KEY_RING_THREADS: if (v != 0 && v != 128 && v != 256) return SPHNSE_E_ARG; P->ring_threads = int(v); return SPHNSE_OK;
        default: return SPHNSE_E_ARG;
    }
}

int sphnse_plan_get(const sphnse_plan* P, int key, double* v) {
    if (!P || !v) return SPHNSE_E_ARG;
    switch (key) {
        case SPHNSE_KEY_PRECISION: *v = P->precision; break;
        case SPHNSE_KEY_NU: *v = P->nu; break;
        case SPHNSE_KEY_OMEGA: *v = P->Omega; break;
        case SPHNSE_KEY_RTOL: *v = P->rtol; break;
        case SPHNSE_KEY_ATOL: *v = P->atol; break;
        case SPHNSE_KEY_MAX_ORDER: *v = P->max_order; break;
        case SPHNSE_KEY_NEWTON_MAX_ITER: *v = P->newton_max; break;
        case SPHNSE_KEY_H_MAX: *v = P->h_max; break;
        case SPHNSE_KEY_BDF: *v = P->bdf; break;
        case SPHNSE_KEY_CORIOLIS_SPLIT: *v = P->coriolis_split; break;
        case SPHNSE_KEY_TIMING_PERIOD: *v = P->timing_period; break;
        case SPHNSE_KEY_RING_THREADS: *v = P->ring_threads; break;
        case SPHNSE_KEY_N_COEFF: *v = P->n_coeff; break;
        case SPHNSE_KEY_L: *v = P->N; break;
        case SPHNSE_KEY_NLAT: *v = P->nlat; break;
        case SPHNSE_KEY_NLON: *v = P->nlon; break;
        case SPHNSE_KEY_SYN_ENTRIES: *v = P->tc.syn_entries; break;
        case SPHNSE_KEY_ANA_ENTRIES: *v = P->tc.ana_entries; break;
        case SPHNSE_KEY_TABLE_BYTES: {
            double b = double(P->tc.tsyn_bytes);
            for (const auto& t : P->tab) b += double(t.bytes);
            *v = b;
            break;
        }
        default: return SPHNSE_E_ARG;
    }
    return SPHNSE_OK;
}

int sphnse_grid_nodes(const sphnse_plan* P, double* theta, double* x, double* s, double* w) {
    if (!P) return SPHNSE_E_ARG;
    const size_t b = size_t(P->nlat) * sizeof(double);
    if (theta) std::memcpy(theta, P->theta.data(), b);
    if (x) std::memcpy(x, P->x.data(), b);
    if (s) std::memcpy(s, P->s.data(), b);
    if (w) std::memcpy(w, P->w.data(), b);
    return SPHNSE_OK;
}

int sphnse_rhs(sphnse_plan* P, double t, const double* alpha, const double* forcing, double* out) {
    (void)t;
    if (!P || !alpha || !out || alpha == out) return SPHNSE_E_ARG;
    return rhs_device(P, alpha, forcing, out);
}

int sphnse_grid_fields(sphnse_plan* P, const double* alpha, double* zeta, double* uth, double* uph) {
    if (!P || !alpha) return SPHNSE_E_ARG;
    const int prec = P->precision == SPHNSE_FP64 ? SPHNSE_FP64 : SPHNSE_FP32;
    const bool tc = P->precision == SPHNSE_BF16X3 && tc_supported(P);
    int rc;
    if (tc) {
        if ((rc = launch_synthesis_tc(P, alpha, 0))) return rc;
    } else {
        if ((rc = launch_prep(P, alpha, nullptr, prec))) return rc;
        if ((rc = launch_synthesis(P, 3, prec))) return rc;
    }
    if ((rc = launch_transpose(P, P->d_gsyn, P->d_gsyn_r, P->N + 1, P->nlat, 3, prec))) return rc;
    return launch_ring(P, RING_GRID, prec, nullptr, nullptr, zeta, uth, uph);
}

int sphnse_project(sphnse_plan* P, const double* vth, const double* vph, double* out) {
    if (!P || !vth || !vph || !out) return SPHNSE_E_ARG;
    const int prec = P->precision == SPHNSE_FP64 ? SPHNSE_FP64 : SPHNSE_FP32;
    int rc;
    if ((rc = launch_ring(P, RING_PROJECT, prec, vth, vph, nullptr, nullptr, nullptr))) return rc;
    if ((rc = launch_transpose(P, P->d_gana_r, P->d_gana, P->nlat, P->N + 1, 2, prec))) return rc;
    const bool tc = P->precision == SPHNSE_BF16X3 && tc_supported(P);
    if ((rc = tc ? launch_analysis_tc(P, 2) : launch_analysis(P, 2, prec))) return rc;
    return launch_finish(P, 1, prec, nullptr, nullptr, out);
}

int sphnse_sync(sphnse_plan* P) {
    if (!P) return SPHNSE_E_ARG;
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return SPHNSE_E_CUDA;
    unsigned st = 0;
    if (cudaMemcpy(&st, P->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return SPHNSE_E_CUDA;
    if (st) {
        cudaMemset(P->d_status, 0, sizeof(unsigned));
        return SPHNSE_E_TIMEOUT;
    }
    return SPHNSE_OK;
}

int sphnse_stage_timing(sphnse_plan* P, int enable) {
    if (!P) return SPHNSE_E_ARG;
    if (enable) {
        fold_stage_events(P);
        for (int s = 0; s < SPHNSE_NSTAGES; ++s) {
            P->stage_ms[s] = 0;
            P->stage_n[s] = 0;
            P->stage_calls[s] = 0;
        }
    }
    P->timing = unsigned(enable) & ((1u << SPHNSE_NSTAGES) - 1);
    return SPHNSE_OK;
}

int sphnse_stage_times(sphnse_plan* P, double* ms, long* launches) {
    if (!P) return SPHNSE_E_ARG;
    fold_stage_events(P);
    for (int s = 0; s < SPHNSE_NSTAGES; ++s) {
        if (ms) ms[s] = P->stage_ms[s];
        if (launches) launches[s] = P->stage_n[s];
    }
    return SPHNSE_OK;
}

// host-only helpers (no CUDA): the FP64 precompute, exposed for checks
int sphnse_host_gauss_nodes(int n, double* theta, double* x, double* s, double* w) {
    if (n < 1 || !theta || !x || !s || !w) return SPHNSE_E_ARG;
    gauss_legendre(n, theta, x, s, w);
    return SPHNSE_OK;
}

int sphnse_host_legendre(int Kmax, int m, int np, const double* x, const double* s, double* out) {
    if (Kmax < m || m < 0 || np < 1 || !x || !s || !out) return SPHNSE_E_ARG;
    legendre_column(Kmax, m, np, x, s, out);
    return SPHNSE_OK;
}

}  // extern "C"
