// Internal declarations of libsphnse (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/sphnse.h"

namespace sph {

// ---- index helpers --------------------------------------------------------
// Packed coefficients: m-major, L = max(m,1)..N.
__host__ __device__ inline int packed_off(int N, int m) {
    return m == 0 ? 0 : N + (m - 1) * (N + 1) - (m - 1) * m / 2;
}
__host__ __device__ inline int packed_index(int N, int m, int L) {
    return packed_off(N, m) + L - (m > 0 ? m : 1);
}
inline int n_packed(int N) { return (N + 1) * (N + 2) / 2 - 1; }
// inverse of packed_index: (L, m) of packed entry i (m = 0 holds L = 1..N, then
// order m >= 1 holds L = m..N from N + u (N+1) - u (u+1) / 2, u = m - 1)
__host__ __device__ inline void packed_lm(int N, int i, int& L, int& m) {
    if (i < N) {
        m = 0;
        L = i + 1;
        return;
    }
    const int ip = i - N;
    const float b = float(N) + 0.5f;
    const float disc = b * b - 2.f * float(ip);
    int u = int(b - sqrtf(disc > 0.f ? disc : 0.f));
    auto off = [N](int v) { return v * (N + 1) - v * (v + 1) / 2; };
    while (u > 0 && off(u) > ip) --u;
    while (u < N && off(u + 1) <= ip) ++u;
    m = u + 1;
    L = ip - off(u) + m;
}

// Complex index of (field f, order m, latitude row) in a synthesis output:
// order-major [f][m][row], or latitude-pair-major [f][row / 2][m][row % 2]
// (pairs != 0), the layout the four-step ring kernel reads contiguously.
__host__ __device__ inline size_t gsyn_index(int pairs, int f, int m, int row, int N, int nlat) {
    return pairs ? ((size_t(f) * (nlat / 2) + row / 2) * size_t(N + 1) + m) * 2 + (row & 1)
                 : (size_t(f) * (N + 1) + m) * size_t(nlat) + row;
}

// Extended-degree ("ext") rows: for each m the degrees K = m..N+1 (n_m = N+2-m
// of them), split by the parity of K - m: even rows first (K = m + 2j,
// j < ne(m)), then odd rows (K = m + 1 + 2j, j < no(m)).  Degree N+1 is needed
// by the theta-derivative recombination.
__host__ __device__ inline int ext_off(int N, int m) { return m * (N + 2) - m * (m - 1) / 2; }
__host__ __device__ inline int ext_count(int N, int m) { return N + 2 - m; }
__host__ __device__ inline int ext_even(int N, int m) { return (N + 3 - m) / 2; }
__host__ __device__ inline int ext_odd(int N, int m) { return (N + 2 - m) / 2; }
__host__ __device__ inline int ext_row(int N, int m, int K) {
    int d = K - m;
    return ext_off(N, m) + ((d & 1) ? ext_even(N, m) + (d >> 1) : (d >> 1));
}
inline int n_ext(int N) { return ext_off(N, N + 1); }

// ---- host precompute (host_tables.cpp) ------------------------------------
// Gauss-Legendre rule, nodes north to south: theta, cos, sin, weights.
void gauss_legendre(int n, double* theta, double* x, double* s, double* w);
// Orthonormal associated Legendre functions Pt_K^m(x_p), K = m..Kmax, for
// the np given nodes; out[(K - m) * np + p].  Extended binary exponent inside.
void legendre_column(int Kmax, int m, int np, const double* x, const double* s, double* out);
// Full table in the synthesis layout: out[ext_row(N, m, K) * nh + p] for the nh
// northern nodes (FP64), computed with nthreads host threads.
void legendre_table_syn(int N, int nh, const double* x, const double* s, double* out);

// ---- radix plan of the longitude FFT (2^a 3^b) -----------------------------
struct FFTPlan {
    int n = 0;
    int nstages = 0;
    int radix[24];
};
bool make_fft_plan(int n, FFTPlan* p);

// ---- device tables ----------------------------------------------------------
struct Tables {
    void* syn = nullptr;     // [n_ext][nh]: rows of Pt over northern nodes (synthesis)
    void* ana = nullptr;     // per (m, parity) block [nh][rows] (analysis)
    void* syn_lo = nullptr;  // BF16X3: low parts
    void* ana_lo = nullptr;
    size_t bytes = 0;
    bool built = false;
};

// Instance groups of a batched tcgen05 synthesis (one truncation): B tiles and
// the LPT item schedule (m, latitude tile, group).
struct TcBatch {
    int nb = 0, ng = 0, ngroups = 0, brows = 0, ns = 0, ncta = 0;
    int cs = 1;                        // CTAs per cluster sharing every table tile (multicast)
    unsigned char* btiles = nullptr;   // [group][tile][brows][64] bf16, swizzled
    int4* items = nullptr;             // (m, latitude tile, group, first K tiles) per CTA at c * istride
    int* cnt = nullptr;                // items per CTA
    int istride = 0;
};

// Batched tcgen05 analysis (NF = 2) over nb instances of one truncation:
// items (tile, slots of (block, instance)) and the per-instance S tiles.
struct TcBatchA {
    int nb = 0, nkt = 0, ncta = 0;
    int4* items = nullptr;
    int* off = nullptr;
    int4* slots = nullptr;
    unsigned char* stiles = nullptr;   // [instance][block][kt] 1 KB
};

// Simplified-Newton loop state of one corrector attempt: inputs set when the
// attempt starts (by the host or the step loop's controller), loop state and
// results updated after every iteration by the stopping rule (on the host, or
// in the last block of the graph's Newton update).
struct NewtonCtl {
    double c, nu, omega, thr, rtol, rate;   // inputs (rate: the running contraction estimate)
    int k, maxit, tight, fp64, havrate;
    unsigned arrived;                       // blocks of the Newton update done with this iteration
    double nrm[4], ynorm, oldnrm;           // results / loop state
    int it, its, conv, stop, nonfinite, pad1;
};

// State of the device-side step loop (sphnse_advance as one graph launch):
// the controller's inputs and memory, loaded from the sphnse_state before the
// launch and stored back after it, and the current attempt's parameters that
// the loop's kernels read.
struct StepCtl {
    double rtol, thr, h_max;                 // per call
    int maxk, newton_max, fp64, nsteps;
    double nu, omega;
    double gamma[SPHNSE_MAXK], iga[SPHNSE_MAXK], ec[SPHNSE_MAXK];
    sphnse_step_info* info;                  // nsteps entries (device in the graph, host otherwise) or null
    double t, h, t_end, h_dif, rate, miter_h;  // integrator state (sphnse_state)
    int order, nconhk, havrate, miter_k;
    int done, attempt, nofailed, rejections, newton_total, rhs_evals;
    double h_dif_before;
    int status;                              // SPHNSE_OK, else the error that ended the loop
    int k, do_rescale;                       // the current attempt
    int accept, k_acc;                       // the last attempt was accepted at order k_acc
    double err;                              // its error estimate
    int sum_newton, sum_rejections;          // over the accepted steps of the call
    int phase;                               // ensemble rounds: 0 idle, 1 new attempt next, 2 in Newton
    double h_att;
    double A[SPHNSE_MAXK * SPHNSE_MAXK];     // difference rescaling matrix (do_rescale)
    double g[SPHNSE_MAXK];                   // predictor weights of psi
    NewtonCtl nc;
};

// staging of sphnse_rhs_host: two slots, an upload and a download stream
struct HostIO {
    void* din[2] = {nullptr, nullptr};
    void* dfo[2] = {nullptr, nullptr};
    void* dout[2] = {nullptr, nullptr};
    cudaEvent_t ev_up[2] = {nullptr, nullptr}, ev_rhs[2] = {nullptr, nullptr}, ev_down[2] = {nullptr, nullptr};
    cudaStream_t up = nullptr, down = nullptr;
    long long calls = 0;
    bool ready = false;
    // direct output (a page-locked, device-mapped out_h on the fused
    // tensor-core RHS): the analysis writes F into out_h, and its last CTA
    // writes the call's ticket + 1 to *flag (mapped host memory) after every
    // CTA's writes of F
    volatile unsigned long long* flag = nullptr;
    unsigned long long* dflag = nullptr;   // device address of flag
    unsigned* dcnt = nullptr;              // CTAs of the running analysis done
    long long direct[2] = {-1, -1};        // the last direct-output call of each slot
};

// tcgen05 path state (tensor maps and item schedules, built on first use)
struct TcState {
    void* map_hi = nullptr;      // CUtensorMap of the whole [n_ext][nh] table, global memory
    void* map_lo = nullptr;
    int4* ana_items = nullptr;   // (first row, first piece, piece count, MMA N | first K tile << 16)
    int* ana_off = nullptr;
    int4* ana_pieces = nullptr;  // (m, parity, first item row, end item row)
    int ana_cta = 0;
    int ana_nf = 0;
    bool ana_ready = false;
    // the RHS analysis with the finish in its epilogue: order-aligned tiles
    // in whole order groups per CTA (items and pieces as above, and per item
    // (group's first row, first order, end order, last item of the group))
    int4* anf_items = nullptr;
    int* anf_off = nullptr;
    int4* anf_pieces = nullptr;
    int4* anf_og = nullptr;
    void* anf_map_hi = nullptr;  // 8 maps of the table, boxes of 16 (j + 1) rows
    void* anf_map_lo = nullptr;
    int anf_cta = 0;
    bool anf_ready = false;
    void* smap_hi = nullptr;     // synthesis: tensor maps of the transposed tables
    void* smap_lo = nullptr;
    void* smap_hi_c2 = nullptr;  // the same with boxes of 64 and 32 latitudes (cluster slices)
    void* smap_lo_c2 = nullptr;
    void* smap_hi_c4 = nullptr;
    void* smap_lo_c4 = nullptr;
    std::vector<size_t> tsyn_off;   // element offset of every block in the transposed tables
    void* tsyn_hi = nullptr;     // transposed padded bf16 tables [block][nh][pad8(n)]
    void* tsyn_lo = nullptr;
    int* tile_off = nullptr;     // first B tile of block (m, parity)
    int2* tile_info = nullptr;   // (block, K tile) of every B tile, in tile order
    int ntiles = 0;
    TcBatch single;              // the plan's own instance
    size_t tsyn_bytes = 0;
    bool syn_ready = false;
    // negligible table tiles: first significant synthesis K tile per (block,
    // latitude tile) (the block's tile count if none), [2 (N + 1)][latitude
    // tiles], and max |Pt| per (table row, 64-latitude chunk)
    double syn_entries = 0, ana_entries = 0;   // table entries one launch reads (skip rule applied)
    std::vector<int> syn_kt0_host;
    std::vector<float> chunk_max;
};

}  // namespace sph

struct sphnse_plan {
    int N = 0, nlat = 0, nlon = 0, nh = 0;   // nh = ceil(nlat/2) northern rows
    double nu = 0, Omega = 0;
    int precision = SPHNSE_FP64;
    double rtol = 1e-6, atol = 1e-12, h_max = 1.0;
    int max_order = 5, newton_max = 4, bdf = 0;
    int coriolis_split = 0;      // Coriolis as the diagonal -2 i Omega m / lambda (forward RHS)
    cudaStream_t stream = nullptr;
    int device = 0;
    int n_coeff = 0, n_ext = 0;
    sph::FFTPlan fft;

    std::vector<double> theta, x, s, w;   // host nodes
    std::vector<double> psyn_host;        // FP64 master table, synthesis layout

    // device constants
    double* d_x = nullptr;       // cos(theta_p), nlat
    double* d_s = nullptr;       // sin(theta_p), nlat
    float* d_isin32 = nullptr;   // 1 / sin(theta_p) rounded to FP32, nlat
    double* d_rw = nullptr;      // (2 pi / M) w_p / sin(theta_p), nlat
    double* d_tw = nullptr;      // e^{-2 pi i t / M}, M complex (FP64)
    float* d_tw32 = nullptr;     // same in FP32
    float* d_ftw = nullptr;      // four-step ring kernel twiddles (M = 24 M2), FP32
    int2* d_lm = nullptr;        // (L, m) of each packed entry
    double4_32a* d_prepc = nullptr;  // per ext row (m, K): (lam_K^{1/2}, lam_K^{-1/2}, c_down, c_up)
    float4* d_prepc32 = nullptr; // FP32 copies of the two coefficient tables
    float4* d_finc32 = nullptr;
    double4_32a* d_finc = nullptr;   // per packed (L, m): (lam^{-1/2}, L eps_{L+1,m} lam^{-1/2},
                                 //                     (L+1) eps_{L,m} lam^{-1/2}, lam)

    sph::Tables tab[3];
    sph::TcState tc;

    // workspaces (sized for the largest field counts: 5 synthesis, 3 analysis)
    void* d_bsyn = nullptr;      // [n_ext][2 * 5] (re, im) per field, precision type
    void* d_gsyn = nullptr;      // [5][N+1][nlat] complex (m-major)
    void* d_gana = nullptr;      // [3][N+1][nlat] complex (m-major)
    void* d_hana = nullptr;      // [n_ext][2 * 3]
    void* d_gsyn_r = nullptr;    // latitude-major copies for the ring kernel: [5][nlat][N+1]
    void* d_gana_r = nullptr;    //                                             [3][nlat][N+1]
    double* d_work = nullptr;    // NDF / adjoint vectors (16 x n_coeff complex)
    double* d_grid = nullptr;    // objective: two grid fields (allocated on first use)
    double* d_theta = nullptr;
    double* d_w = nullptr;
    double* d_tmp = nullptr;     // 2 x n_coeff complex scratch for F / J^T w
    int n_cta = 0;               // persistent streaming grid (one CTA per SM)
    int* d_items = nullptr;      // orders m per CTA (LPT schedule on L + 2 - m rows)
    int* d_item_off = nullptr;   // [n_cta + 1]
    unsigned* d_status = nullptr;  // device status word (bounded-wait timeouts)
    unsigned long long* d_norms = nullptr;  // 8 reduction slots
    double* h_norms = nullptr;   // pinned host mirror
    size_t work_bytes = 0;

    // optional per-stage CUDA-event timing on the plan's stream
    unsigned timing = 0;         // bit mask of timed stages
    int timing_period = 1;       // record every timing_period-th launch of a timed stage
    int ring_threads = 0;        // four-step ring kernel: 0 chooses, 128 or 256 threads per G rings
    // set for one direct-output sphnse_rhs_host call: the RHS analysis reports completion
    unsigned* done_cnt = nullptr;
    unsigned long long* done_flag = nullptr;
    unsigned long long done_ticket = 0;
    int nsm = 1;                 // SMs of the plan's device
    long stage_calls[8] = {};    // launches seen per stage while timed
    bool stage_rec[8] = {};      // the current launch of the stage is recorded
    std::vector<cudaEvent_t> ev[SPHNSE_NSTAGES];
    sph::HostIO hio;
    // device-side Newton loop (sphnse_step, sphnse_replay_step)
    cudaGraphExec_t ng_exec = nullptr;
    const void* ng_key[4] = {nullptr, nullptr, nullptr, nullptr};   // alpha, dif, forcing, precision + split
    double ng_nu = 0, ng_omega = 0;
    bool ng_failed = false;              // capture not possible here: the host loop runs
    sph::NewtonCtl* d_ctl = nullptr;
    sph::NewtonCtl* h_ctl = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream for capturing the loop body
    // device-side step loop (sphnse_advance, sphnse_step): outer WHILE over
    // attempts, the Newton WHILE nested in its body
    cudaGraphExec_t sg_exec = nullptr;
    const void* sg_key[4] = {nullptr, nullptr, nullptr, nullptr};
    double sg_nu = 0, sg_omega = 0;
    bool sg_failed = false;
    sph::StepCtl* d_step = nullptr;
    sph::StepCtl* h_step = nullptr;      // pinned
    sphnse_step_info* d_info = nullptr;
    sphnse_step_info* h_info = nullptr;  // pinned
    int info_cap = 0;
    int ev_used[SPHNSE_NSTAGES] = {0};
    double stage_ms[SPHNSE_NSTAGES] = {0};
    long stage_n[SPHNSE_NSTAGES] = {0};
};

namespace sph {

// ---- launchers (kernels in *.cu) ------------------------------------------
enum RingMode { RING_RHS = 0, RING_GRID = 1, RING_PROJECT = 2, RING_ADJOINT = 3 };

// prep: coefficient sets for synthesis.  nsets fields from alpha (3: zeta,
// theta, phi) and optionally 2 more (theta, phi) from beta scaled by 1/s_m.
int launch_prep(sphnse_plan* P, const double* alpha, const double* beta, int prec);
// pairs != 0: write the latitude-pair-major layout of gsyn_index
int launch_synthesis(sphnse_plan* P, int nfields, int prec, int pairs = 0);
int launch_ring(sphnse_plan* P, int mode, int prec, const double* gin0, const double* gin1,
                double* gout0, double* gout1, double* gout2);
int launch_analysis(sphnse_plan* P, int nfields, int prec);
// in [nf][R][Cn] -> out [nf][Cn][R] (complex entries of the precision's type)
int launch_transpose(sphnse_plan* P, const void* in, void* out, int R, int Cn, int nf, int prec);
// finish: kind 0 = RHS (F = f - nu lam alpha - N), 1 = projection (N),
// 2 = adjoint (out = -nu lam w - s_m (N_X + lam^{1/2} H_rho))
int launch_finish(sphnse_plan* P, int kind, int prec, const double* alpha,
                  const double* forcing, double* out);

int ensure_tables(sphnse_plan* P, int prec);
bool stream_ok(const sphnse_plan* P, int prec);
int launch_synthesis_stream(sphnse_plan* P, int nfields, int prec, int pairs = 0);
bool tc_supported(const sphnse_plan* P);
int launch_analysis_tc(sphnse_plan* P, int nfields);
// the RHS's analysis (two product fields) with the recombination and update
// of the finish step in the epilogue: F = forcing - nu lambda alpha - N
int launch_analysis_finish_tc(sphnse_plan* P, const double* alpha, const double* forcing, double* out);
// true when the RHS runs as the three fused tensor-core kernels (the
// synthesis builds its coefficient tiles, the analysis runs the finish)
bool tc_rhs_fused(sphnse_plan* P);
// coefficient prep and synthesis of the plan's own instance (alpha: packed
// coefficients on the device)
int launch_synthesis_tc(sphnse_plan* P, const double* alpha, int pairs);
// batched tcgen05 synthesis over nb instances of P's truncation (ensembles)
int tc_setup_synthesis(sphnse_plan* P);
// instance groups of at most ngmax (<= 9) instances, at most nsmax (<= 6)
// pipeline stages (fewer when the shared memory does not hold them)
int tc_batch_init(sphnse_plan* P, int nb, TcBatch* B, int ngmax = 9, int nsmax = 6, int cs = 1);
void tc_batch_free(TcBatch* B);
int launch_prep_tc_batch(sphnse_plan* P, const TcBatch& B, const double* alpha);
int launch_synthesis_tc_batch(sphnse_plan* P, const TcBatch& B, float* gsyn, size_t sg_floats, int pairs,
                              const double* alpha = nullptr);
int tc_setup_analysis(sphnse_plan* P, int nf);
int tc_batch_ana_init(sphnse_plan* P, int nb, TcBatchA* B);
void tc_batch_ana_free(TcBatchA* B);
int launch_analysis_tc_batch(sphnse_plan* P, const TcBatchA& B, const float* gana, size_t sa_floats, float* hana,
                             size_t sh_floats);
// batched FP32 passes over instances of one truncation (ensemble)
int launch_prep32_batch(sphnse_plan* P, int nb, const double* alpha, float* bsyn, size_t bstride);
int launch_synthesis_stream_batch(sphnse_plan* P, const int* items, const int* item_off, int ncta,
                                  const float* bsyn, size_t sb, float* gsyn, size_t sg, int pairs);
int launch_ring_batch(sphnse_plan* P, int nb, const float* gsyn_r, size_t sgs, float* gana_r, size_t sga);
// four-step FP32 RHS ring kernel on the order-major buffers (M = 24 M2, M2 = 4..64, nlat even)
int ring4_m2(int nlon, int nlat);
bool ring4_ok(const sphnse_plan* P);
std::vector<float> ring4_twiddles(int nlon);
int launch_ring4(sphnse_plan* P, int nb, const float* gsyn, size_t sgs, float* gana, size_t sga, int pairs);
int launch_analysis_stream_batch(sphnse_plan* P, const int* items, const int* item_off, int ncta,
                                 const float* gana, size_t sa, float* hana, size_t sh);
int launch_finish32_batch(sphnse_plan* P, int nb, const float* hana, size_t hstride, const double* alpha,
                          double* out, const double* nu_inst);
void tc_free(sphnse_plan* P);
void host_io_free(sphnse_plan* P);
int launch_analysis_stream(sphnse_plan* P, int nfields, int prec);
void stage_begin(sphnse_plan* P, int stage);
void stage_end(sphnse_plan* P, int stage);
int check_cuda(cudaError_t e);

// Ask once per kernel for the largest shared-memory carveout.  An SM runs
// CTAs of different kernels together only under one L1/shared split: when a
// small kernel (no shared memory) prefers the default split, the next
// kernel's CTAs that need ~200 KB cannot start on an SM until it drains,
// which defeats the early launch below.
void prefer_max_smem(const void* kernel);

// Raise the kernel's dynamic shared-memory cap to at least `bytes` and never
// lower it.  One kernel is launched with different sizes by different
// plans, ensemble buckets and tuned shapes, and launches recorded in graphs
// are checked against the cap as it stands when they run (a profiler
// replays graph nodes one by one): the cap must cover every size ever used.
void allow_dynamic_smem(const void* kernel, size_t bytes);

// Launch with programmatic stream serialisation (the kernel calls pdl_wait()
// before it reads what its predecessor on the stream wrote).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                              Args... args) {
    prefer_max_smem(reinterpret_cast<const void*>(kernel));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Programmatic launch only for a grid that fits one wave (at most one CTA
// per SM): a dependent launched early holds SM slots while it waits, which
// slows a predecessor that still has CTAs to place.  The small grids of a
// latency-bound plan gain the launch overlap; large grids launch normally.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl_small(int n_sm, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t stream, Args... args) {
    if (long(grid.x) * grid.y * grid.z <= n_sm) return launch_pdl(kernel, grid, block, smem, stream, args...);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// whole pipelines
int rhs_device(sphnse_plan* P, const double* alpha, const double* forcing, double* out);
int rhs_adjoint_device(sphnse_plan* P, const double* alpha, const double* w, double* out);

}  // namespace sph
