// Persistent streaming Legendre kernels (CUDA cores, FP64 or FP32).
//
// The per-order Legendre sums of the RHS (Sec. 4.2; synthesis of the fields
// of Eq. (app_soln_rep) and (vort_app), analysis = the discrete projection of
// Eq. (disc_vec_orth_proj)) stream the table Pt_K^m(x_p) once per pass; the
// table (>= 200 MB at L = 511) is far larger than L2, so the kernels are
// HBM-bound.  Design:
//   * one CTA per SM, persistent; the orders m are dealt to CTAs by a host
//     LPT schedule on the per-order row counts (L + 2 - m rows each);
//   * a producer warp streams rows with 1-D bulk async copies (TMA engine)
//     into an NST-stage shared-memory ring (evict-first L2 policy, so the
//     L2-resident intermediates survive); each stage holds HR even-parity and
//     HR odd-parity rows (K - m even / odd) of the current order;
//   * consumer warps wait on the stage's full mbarrier, compute, and release
//     it through its empty mbarrier;
//   * synthesis: two thread groups (even rows -> E, odd rows -> O) each own V
//     consecutive latitudes per thread, epilogue north = E + O, south = E - O;
//   * analysis: teams of warps take whole stages; a warp reduces 4 rows at a
//     time over the latitudes (lanes split p) with a transpose-reduction.
// Table layout [ext row][nh]: row (m, K) holds Pt_K^m at the nh northern nodes.
#include <cuda_runtime.h>

#include "internal.h"
#include "ptx.cuh"

namespace sph {

// pipeline depth: 6 stages of 24 KB for FP32; 4 for FP64 (compute bound and
// tighter on shared memory)
template <typename T> __host__ __device__ constexpr int nst() { return sizeof(T) == 4 ? 6 : 4; }

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ void vload(const T* p, T* out) {
    using VT = typename Vec<T>::type;
    const VT v = *reinterpret_cast<const VT*>(p);
    const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
    for (int i = 0; i < Vec<T>::n; ++i) out[i] = e[i];
}

struct StreamArgs {
    const void* table;   // [n_ext][nh]
    const void* bsyn;    // synthesis coefficient sets [n_ext][2 NF]
    void* gsyn;          // [NF][N+1][nlat] complex (m-major)
    const void* gana;    // [NF][N+1][nlat] complex (m-major)
    void* hana;          // [n_ext][2 NF]
    const double* sinth;
    const int* items;    // orders m, grouped per CTA
    const int* item_off; // [gridDim + 1]
    unsigned* status;
    int N, nh, nlat;
    // batches: an item v stands for instance v / (N+1) and order v % (N+1);
    // per-instance strides (elements) of bsyn, gsyn, gana, hana
    size_t sb, sg, sa, sh;
    int pairs;           // gsyn layout (gsyn_index)
};

// chunk c of order m: rows [c HR, c HR + HR) of the even and of the odd block
__device__ __forceinline__ void chunk_rows(int ne, int no, int c, int HR, int* cnt_e, int* cnt_o) {
    int ce = ne - c * HR, co = no - c * HR;
    *cnt_e = ce < 0 ? 0 : (ce > HR ? HR : ce);
    *cnt_o = co < 0 ? 0 : (co > HR ? HR : co);
}

// Producer: lane 0 of warp 0 walks the CTA's (order, chunk) sequence.
template <typename T, int HR>
__device__ void produce(const StreamArgs& a, T* stages, uint64_t* full, uint64_t* empty, volatile int* abort,
                        int n_items_begin, int n_items_end) {
    const uint64_t pol = policy_evict_first();
    const T* tab = reinterpret_cast<const T*>(a.table);
    const size_t rowb = size_t(a.nh) * sizeof(T);
    int it = 0;
    for (int ii = n_items_begin; ii < n_items_end; ++ii) {
        const int m = a.items[ii] % (a.N + 1);
        const int ne = ext_even(a.N, m), no = ext_odd(a.N, m), e0 = ext_off(a.N, m);
        const int nch = ((ne > no ? ne : no) + HR - 1) / HR;
        for (int c = 0; c < nch; ++c, ++it) {
            const int s = it % nst<T>();
            const uint32_t ph = (it / nst<T>()) & 1;
            if (it >= nst<T>() && !mbar_wait(&empty[s], ph ^ 1, abort, a.status)) continue;
            if (*abort) continue;
            int ce, co;
            chunk_rows(ne, no, c, HR, &ce, &co);
            T* dst = stages + size_t(s) * 2 * HR * a.nh;
            mbar_arrive_expect_tx(&full[s], uint32_t((ce + co) * rowb));
            if (ce) bulk_g2s(dst, tab + size_t(e0 + c * HR) * a.nh, uint32_t(ce * rowb), &full[s], pol);
            if (co) bulk_g2s(dst + size_t(HR) * a.nh, tab + size_t(e0 + ne + c * HR) * a.nh, uint32_t(co * rowb),
                             &full[s], pol);
        }
    }
    // wait for the copies still in flight before leaving (bounded)
    const int last = it;
    for (int k = last - nst<T>(); k < last; ++k) {
        if (k < 0) continue;
        mbar_wait(&full[k % nst<T>()], (k / nst<T>()) & 1, abort, a.status);
    }
}

// ---------------------------------------------------------------------------
// synthesis

template <typename T, int NF, int HR>
__global__ void __launch_bounds__(512, 1) k_syn_stream(StreamArgs a) {
    constexpr int V = Vec<T>::n;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    constexpr int NST = nst<T>();
    uint64_t* empty = full + NST;
    volatile int* abort = reinterpret_cast<volatile int*>(empty + NST);
    T* stages = reinterpret_cast<T*>(smem + 128);
    const int nh = a.nh, N = a.N, nlat = a.nlat;
    T* Bsm = stages + size_t(NST) * 2 * HR * nh;                 // 2 x [N+2][2 NF]
    T* red = Bsm + size_t(2) * (N + 2) * 2 * NF;                  // [nh][2 NF]
    const int tpg = (blockDim.x - 32) / 2;                        // threads per group
    const int n_cwarps = (blockDim.x - 32) / 32;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], n_cwarps);
        }
        *abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    pdl_launch();
    const int ib = a.item_off[blockIdx.x], iend = a.item_off[blockIdx.x + 1];
    if (threadIdx.x < 32) {
        // the tables do not depend on the predecessor: stream them right away
        if (threadIdx.x == 0) produce<T, HR>(a, stages, full, empty, abort, ib, iend);
        return;
    }
    pdl_wait();
    const int ct = threadIdx.x - 32;
    const int g = ct / tpg;               // 0: even rows, 1: odd rows
    const int p0 = (ct % tpg) * V;
    const bool act = p0 < nh;
    const int ncons = blockDim.x - 32;
    const T* bsyn = reinterpret_cast<const T*>(a.bsyn);
    T* gsyn = reinterpret_cast<T*>(a.gsyn);
    int it = 0;
    for (int ii = ib; ii < iend; ++ii) {
        const int inst = a.items[ii] / (N + 1), m = a.items[ii] % (N + 1);
        const int ne = ext_even(N, m), no = ext_odd(N, m), e0 = ext_off(N, m), cnt = ne + no;
        T* B = Bsm + size_t(ii & 1) * (N + 2) * 2 * NF;
        const T* bsrc = bsyn + inst * a.sb;
        T* gdst = gsyn + inst * a.sg;
        for (int i = ct; i < cnt * 2 * NF; i += ncons) B[i] = bsrc[size_t(e0) * 2 * NF + i];
        named_bar_sync(1, ncons);
        T acc[V][2 * NF];
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
            for (int f = 0; f < 2 * NF; ++f) acc[v][f] = T(0);
        const int nch = ((ne > no ? ne : no) + HR - 1) / HR;
        for (int c = 0; c < nch; ++c, ++it) {
            const int s = it % NST;
            const bool ok = mbar_wait(&full[s], (it / NST) & 1, abort, a.status);
            int ce, co;
            chunk_rows(ne, no, c, HR, &ce, &co);
            const int nrow = g ? co : ce;
            if (ok && act) {
                const T* st = stages + (size_t(s) * 2 + g) * HR * nh + p0;
                const T* bb = B + size_t((g ? ne : 0) + c * HR) * 2 * NF;
#pragma unroll 2
                for (int r = 0; r < nrow; ++r) {
                    T pv[V];
                    vload(st + size_t(r) * nh, pv);
                    const T* b = bb + r * 2 * NF;
#pragma unroll
                    for (int f = 0; f < 2 * NF; ++f) {
                        const T bf = b[f];
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v][f] = fma(pv[v], bf, acc[v][f]);
                    }
                }
            }
            __syncwarp();
            if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[s]);
        }
        // epilogue: odd group hands O over through shared memory
        if (g == 1 && act)
#pragma unroll
            for (int v = 0; v < V; ++v)
#pragma unroll
                for (int f = 0; f < 2 * NF; ++f) red[(p0 + v) * 2 * NF + f] = acc[v][f];
        named_bar_sync(1, ncons);
        if (g == 0 && act && !*abort) {
            const T mm = T(m);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int p = p0 + v;
                if (p >= nh) break;
                const T inv_s = T(1.0 / a.sinth[p]);
#pragma unroll
                for (int hemi = 0; hemi < 2; ++hemi) {
                    const int row = hemi == 0 ? p : nlat - 1 - p;
                    if (hemi == 1 && row == p) break;
                    const T sg = hemi == 0 ? T(1) : T(-1);
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const T gr = acc[v][2 * f] + sg * red[p * 2 * NF + 2 * f];
                        const T gi = acc[v][2 * f + 1] + sg * red[p * 2 * NF + 2 * f + 1];
                        T o0, o1;
                        if (f == 0) { o0 = gr; o1 = gi; }
                        else if (f == 1 || f == 3) { o0 = -mm * gi * inv_s; o1 = mm * gr * inv_s; }
                        else { o0 = -gr * inv_s; o1 = -gi * inv_s; }
                        T* d = gdst + gsyn_index(a.pairs, f, m, row, N, nlat) * 2;
                        d[0] = o0;
                        d[1] = o1;
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// analysis

// Transpose-reduction of NV per-lane partial sums across a warp: afterwards
// lane l holds the total of index (NV == 32 ? l : l >> 1).
template <typename T, int NV>
__device__ __forceinline__ T transpose_reduce(T* v) {
    const int lane = threadIdx.x & 31;
    int n = NV;
#pragma unroll
    for (int mask = 16; mask >= 1; mask >>= 1) {
        if (n == 1) {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], mask);
            continue;
        }
        const int half = n / 2;
        const bool b = (lane & mask) != 0;
#pragma unroll
        for (int i = 0; i < NV / 2; ++i) {
            if (i < half) {
                const T keep = b ? v[half + i] : v[i];
                const T send = b ? v[i] : v[half + i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
            }
        }
        n = half;
    }
    return v[0];
}

template <typename T, int NF, int HR, int NTEAM>
__global__ void __launch_bounds__(288, 1) k_ana_stream(StreamArgs a) {
    constexpr int V = Vec<T>::n;
    constexpr int QPS = 2 * HR / 4;               // row quads per stage = warps per team
    constexpr int NVR = 4 * 2 * NF;               // values per lane per quad
    constexpr int NV = NVR <= 16 ? 16 : 32;
    constexpr int FS = NV / 4;                    // slot stride per row in the reduced index
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    constexpr int NST = nst<T>();
    uint64_t* empty = full + NST;
    volatile int* abort = reinterpret_cast<volatile int*>(empty + NST);
    T* stages = reinterpret_cast<T*>(smem + 128);
    const int nh = a.nh, N = a.N, nlat = a.nlat;
    T* Ssm = stages + size_t(NST) * 2 * HR * nh;   // 2 buffers x 2 parities x [nh][2 NF]
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], QPS);
        }
        *abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    pdl_launch();
    const int ib = a.item_off[blockIdx.x], iend = a.item_off[blockIdx.x + 1];
    if (threadIdx.x < 32) {
        // the tables do not depend on the predecessor: stream them right away
        if (threadIdx.x == 0) produce<T, HR>(a, stages, full, empty, abort, ib, iend);
        return;
    }
    pdl_wait();
    const int ct = threadIdx.x - 32, ncons = blockDim.x - 32;
    const int warp = ct / 32, lane = ct & 31;
    const int team = warp / QPS, q = warp % QPS;
    const int par = (q * 4) / HR;                 // quad -> parity block
    const int r0 = (q * 4) % HR;                  // first row of the quad in its block
    const T* gana = reinterpret_cast<const T*>(a.gana);
    T* hana = reinterpret_cast<T*>(a.hana);
    int it = 0;
    for (int ii = ib; ii < iend; ++ii) {
        const int inst = a.items[ii] / (N + 1), m = a.items[ii] % (N + 1);
        const int ne = ext_even(N, m), no = ext_odd(N, m), e0 = ext_off(N, m);
        const T* gsrc = gana + inst * a.sa;
        T* hdst = hana + inst * a.sh;
        // S is field-major: S[par][f][p] (par 0: G(p) + G(p'), 1: G(p) - G(p'))
        // so that a lane's V consecutive latitudes are one conflict-free vector load
        T* S = Ssm + size_t(ii & 1) * 2 * nh * 2 * NF;
        for (int i = ct; i < nh * NF; i += ncons) {
            const int f = i / nh, p = i % nh, pr = nlat - 1 - p;
            const T* ga = gsrc + ((size_t(f) * (N + 1) + m) * nlat + p) * 2;
            T ar = ga[0], ai = ga[1], br = T(0), bi = T(0);
            if (pr != p) {
                const T* gb = gsrc + ((size_t(f) * (N + 1) + m) * nlat + pr) * 2;
                br = gb[0];
                bi = gb[1];
            }
            S[size_t(2 * f) * nh + p] = ar + br;
            S[size_t(2 * f + 1) * nh + p] = ai + bi;
            S[size_t(2 * NF + 2 * f) * nh + p] = ar - br;
            S[size_t(2 * NF + 2 * f + 1) * nh + p] = ai - bi;
        }
        named_bar_sync(1, ncons);
        const int nch = ((ne > no ? ne : no) + HR - 1) / HR;
        for (int c = 0; c < nch; ++c, ++it) {
            if (it % NTEAM != team) continue;
            const int s = it % NST;
            const bool ok = mbar_wait(&full[s], (it / NST) & 1, abort, a.status);
            int ce, co;
            chunk_rows(ne, no, c, HR, &ce, &co);
            const int nrow = (par ? co : ce) - r0;   // rows of this quad present
            if (ok && nrow > 0) {
                T acc[NV];
#pragma unroll
                for (int i = 0; i < NV; ++i) acc[i] = T(0);
                const T* st = stages + (size_t(s) * 2 + par) * HR * nh + size_t(r0) * nh;
                const T* Sp = S + size_t(par) * nh * 2 * NF;
                for (int p = lane * V; p < nh; p += 32 * V) {
                    T pv[4][V];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        if (r < nrow) vload(st + size_t(r) * nh + p, pv[r]);
                        else
#pragma unroll
                            for (int v = 0; v < V; ++v) pv[r][v] = T(0);
                    }
#pragma unroll
#pragma unroll
                    for (int f = 0; f < 2 * NF; ++f) {
                        T sf[V];
                        vload(Sp + size_t(f) * nh + p, sf);
#pragma unroll
                        for (int v = 0; v < V; ++v)
#pragma unroll
                            for (int r = 0; r < 4; ++r) acc[r * FS + f] = fma(pv[r][v], sf[v], acc[r * FS + f]);
                    }
                }
                const T tot = transpose_reduce<T, NV>(acc);
                const int idx = NV == 32 ? lane : (lane >> 1);
                const int r = idx / FS, f = idx % FS;
                const bool writer = (NV == 32 || (lane & 1) == 0) && f < 2 * NF && r < nrow;
                if (writer && !*abort) {
                    const int row = e0 + (par ? ne : 0) + c * HR + r0 + r;
                    hdst[size_t(row) * 2 * NF + f] = tot;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
    }
}

// ---------------------------------------------------------------------------
// host launchers

template <typename T>
static constexpr int half_rows() { return sizeof(T) == 4 ? 8 : 4; }

bool stream_ok(const sphnse_plan* P, int prec) {
    const int V = prec == SPHNSE_FP64 ? 2 : 4;
    return P->d_items != nullptr && P->nh % V == 0 && P->nh >= 32;
}

template <typename T, int NF>
static int syn_stream_t(sphnse_plan* P, int pairs) {
    constexpr int HR = half_rows<T>();
    constexpr int V = Vec<T>::n;
    const int tpg = ((P->nh / V + 31) / 32) * 32;
    const int threads = 32 + 2 * tpg;
    if (threads > 512) return SPHNSE_E_UNSUPPORTED;
    constexpr int NST = nst<T>();
    const size_t sm = 128 + sizeof(T) * (size_t(NST) * 2 * HR * P->nh + size_t(2) * (P->N + 2) * 2 * NF +
                                         size_t(P->nh) * 2 * NF);
    if (sm > 227 * 1024) return SPHNSE_E_UNSUPPORTED;
    allow_dynamic_smem(reinterpret_cast<const void*>(k_syn_stream<T, NF, HR>), sm);
    StreamArgs a{P->tab[sizeof(T) == 8 ? SPHNSE_FP64 : SPHNSE_FP32].syn, P->d_bsyn, P->d_gsyn, nullptr, nullptr,
                 P->d_s, P->d_items, P->d_item_off, P->d_status, P->N, P->nh, P->nlat, 0, 0, 0, 0, pairs};
    stage_begin(P, SPHNSE_STAGE_SYNTHESIS);
    launch_pdl(k_syn_stream<T, NF, HR>, dim3(P->n_cta), dim3(threads), sm, P->stream, a);
    stage_end(P, SPHNSE_STAGE_SYNTHESIS);
    return check_cuda(cudaGetLastError());
}

template <typename T, int NF>
static int ana_stream_t(sphnse_plan* P) {
    constexpr int HR = half_rows<T>();
    constexpr int QPS = 2 * HR / 4;
    constexpr int NTEAM = 8 / QPS;
    const int threads = 32 + 32 * QPS * NTEAM;
    constexpr int NST = nst<T>();
    const size_t sm = 128 + sizeof(T) * (size_t(NST) * 2 * HR * P->nh + size_t(2) * 2 * P->nh * 2 * NF);
    if (sm > 227 * 1024) return SPHNSE_E_UNSUPPORTED;
    allow_dynamic_smem(reinterpret_cast<const void*>(k_ana_stream<T, NF, HR, NTEAM>), sm);
    StreamArgs a{P->tab[sizeof(T) == 8 ? SPHNSE_FP64 : SPHNSE_FP32].syn, nullptr, nullptr, P->d_gana, P->d_hana,
                 P->d_s, P->d_items, P->d_item_off, P->d_status, P->N, P->nh, P->nlat, 0, 0, 0, 0, 0};
    stage_begin(P, SPHNSE_STAGE_ANALYSIS);
    launch_pdl(k_ana_stream<T, NF, HR, NTEAM>, dim3(P->n_cta), dim3(threads), sm, P->stream, a);
    stage_end(P, SPHNSE_STAGE_ANALYSIS);
    return check_cuda(cudaGetLastError());
}

int launch_synthesis_stream(sphnse_plan* P, int nfields, int prec, int pairs) {
    if (prec == SPHNSE_FP64)
        return nfields == 5 ? syn_stream_t<double, 5>(P, pairs) : syn_stream_t<double, 3>(P, pairs);
    return nfields == 5 ? syn_stream_t<float, 5>(P, pairs) : syn_stream_t<float, 3>(P, pairs);
}

int launch_analysis_stream(sphnse_plan* P, int nfields, int prec) {
    if (prec == SPHNSE_FP64) return nfields == 3 ? ana_stream_t<double, 3>(P) : ana_stream_t<double, 2>(P);
    return nfields == 3 ? ana_stream_t<float, 3>(P) : ana_stream_t<float, 2>(P);
}

// FP32 batched streaming passes over instances (items = inst * (N+1) + m)
int launch_synthesis_stream_batch(sphnse_plan* P, const int* items, const int* item_off, int ncta,
                                  const float* bsyn, size_t sb, float* gsyn, size_t sg, int pairs) {
    constexpr int HR = half_rows<float>();
    constexpr int NST = nst<float>();
    const int tpg = ((P->nh / 4 + 31) / 32) * 32;
    const int threads = 32 + 2 * tpg;
    const size_t sm = 128 + sizeof(float) * (size_t(NST) * 2 * HR * P->nh + size_t(2) * (P->N + 2) * 6 +
                                             size_t(P->nh) * 6);
    if (threads > 512 || sm > 227 * 1024 || !stream_ok(P, SPHNSE_FP32)) return SPHNSE_E_UNSUPPORTED;
    allow_dynamic_smem(reinterpret_cast<const void*>(k_syn_stream<float, 3, HR>), sm);
    StreamArgs a{P->tab[SPHNSE_FP32].syn, bsyn, gsyn, nullptr, nullptr, P->d_s, items, item_off, P->d_status,
                 P->N, P->nh, P->nlat, sb, sg, 0, 0, pairs};
    stage_begin(P, SPHNSE_STAGE_SYNTHESIS);
    launch_pdl(k_syn_stream<float, 3, HR>, dim3(ncta), dim3(threads), sm, P->stream, a);
    stage_end(P, SPHNSE_STAGE_SYNTHESIS);
    return check_cuda(cudaGetLastError());
}

int launch_analysis_stream_batch(sphnse_plan* P, const int* items, const int* item_off, int ncta,
                                 const float* gana, size_t sa, float* hana, size_t sh) {
    constexpr int HR = half_rows<float>();
    constexpr int QPS = 2 * HR / 4;
    constexpr int NTEAM = 8 / QPS;
    constexpr int NST = nst<float>();
    const int threads = 32 + 32 * QPS * NTEAM;
    const size_t sm = 128 + sizeof(float) * (size_t(NST) * 2 * HR * P->nh + size_t(2) * 2 * P->nh * 4);
    if (sm > 227 * 1024 || !stream_ok(P, SPHNSE_FP32)) return SPHNSE_E_UNSUPPORTED;
    allow_dynamic_smem(reinterpret_cast<const void*>(k_ana_stream<float, 2, HR, NTEAM>), sm);
    StreamArgs a{P->tab[SPHNSE_FP32].syn, nullptr, nullptr, gana, hana, P->d_s, items, item_off, P->d_status,
                 P->N, P->nh, P->nlat, 0, 0, sa, sh, 0};
    stage_begin(P, SPHNSE_STAGE_ANALYSIS);
    launch_pdl(k_ana_stream<float, 2, HR, NTEAM>, dim3(ncta), dim3(threads), sm, P->stream, a);
    stage_end(P, SPHNSE_STAGE_ANALYSIS);
    return check_cuda(cudaGetLastError());
}

}  // namespace sph
